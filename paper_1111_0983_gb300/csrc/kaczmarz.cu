// Kaczmarz comparison smoother (Sec. 3.3, "Comparison with the Kaczmarz and
// the block relaxations"): after the Gauss-Seidel sweep over the inside
// nodes, lambda sweeps of Kaczmarz steps u += (b_j - <l_j, u>) / ||l_j||^2 l_j
// over the ghost equations and the band's inside equations.  The rows are
// ordered by the colour (i mod 5) + 5 (j mod 5) of their node; a row's
// support lies within 2 nodes of its node, so the rows of one colour share no
// unknown and a colour is one launch, a thread a row.  Plain FP64, 2D.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "gcmg_internal.h"
#include "kernels.h"

namespace gcmg {
namespace {

// Row of an inside node p, scaled by h^2: 4 u_p - (its 4 neighbours) = h^2 f_p;
// row of ghost q: sum_k w_k u_k = g_q.  Products rounded on their own, sums
// in the order written (as the oracle's kaczmarz_row).
__global__ void __launch_bounds__(256) k_kaczmarz(LevelView<double> v, const int32_t *__restrict__ rows, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t x = rows[k];
    double *u = v.u;
    if (x >= 0) {
        const int64_t p = x;
        const double s = (u[p + v.s0] + u[p - v.s0]) + (u[p + 1] + u[p - 1]);
        const double r = (__dmul_rn(v.h2, v.f[p]) + s) - 4.0 * u[p];
        const double t = r / 20.0;
        u[p] = u[p] + 4.0 * t;
        u[p + v.s0] = u[p + v.s0] - t;
        u[p - v.s0] = u[p - v.s0] - t;
        u[p + 1] = u[p + 1] - t;
        u[p - 1] = u[p - 1] - t;
        return;
    }
    const int q = -x - 1;
    double s = 0.0, n2 = 0.0;
#pragma unroll
    for (int a = 0; a < 9; a++) {
        const double w = v.gw[(int64_t)a * v.ng + q];
        if (w == 0.0) continue;   // a stencil slot the ghost does not use
        s = s + __dmul_rn(w, u[v.gstn[(int64_t)a * v.ng + q]]);
        n2 = n2 + __dmul_rn(w, w);
    }
    const double t = (v.gg[q] - s) / n2;
#pragma unroll
    for (int a = 0; a < 9; a++) {
        const double w = v.gw[(int64_t)a * v.ng + q];
        if (w == 0.0) continue;
        const int32_t st = v.gstn[(int64_t)a * v.ng + q];
        u[st] = u[st] + __dmul_rn(t, w);
    }
}

}  // namespace

void launch_kaczmarz(const LevelView<double> &v, const int32_t *rows, const std::vector<int32_t> &off, int sweeps,
                     cudaStream_t s) {
    for (int m = 0; m < sweeps; m++)
        for (size_t c = 0; c + 1 < off.size(); c++) {
            const int n = off[c + 1] - off[c];
            if (n <= 0) continue;
            g_launches++;
            k_kaczmarz<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, rows + off[c], n);
        }
}

}  // namespace gcmg
