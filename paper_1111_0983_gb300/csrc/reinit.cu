// Reinitialisation of a level set towards a signed distance function
// (Eq. sdf, Sec. 2.1): phi_t = sgn(phi0) (1 - |grad phi|), explicit steps of
// dt = h / d from phi = phi0.  The discretisation is the Godunov upwinding of
// |grad phi| with the sign of phi0 and, at nodes with an axis neighbour across
// the zero set of phi0, the subcell fix that moves phi towards
// h phi0 / Delta phi0 (Delta phi0: the largest centred or one-sided
// difference of phi0 over the axes), which keeps the zero set where phi0 has
// it.  Outside the box a node's own value is used.  One thread per node.
#include <cuda_runtime.h>

#include <cstdint>

#include "gcmg.h"

namespace {

template <int D>
__global__ void __launch_bounds__(256) k_reinit_step(int n, int64_t nn, const double *__restrict__ p0,
                                                     const double *__restrict__ p, double *__restrict__ q) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const double h = 2.0 / (n - 1), dt = h / D;
    int j[D];
    int64_t st[D];
    {
        int64_t rem = i, s = 1;
        for (int a = D - 1; a >= 0; a--) {
            st[a] = s;
            s *= n;
        }
        for (int a = 0; a < D; a++) {
            j[a] = (int)(rem / st[a]);
            rem -= (int64_t)j[a] * st[a];
        }
    }
    const double pi = p[i], p0i = p0[i];
    const double s = (double)((p0i > 0.0) - (p0i < 0.0));
    bool near = false;
    double dmax = 0.0, g = 0.0;
#pragma unroll
    for (int a = 0; a < D; a++) {
        const int64_t im = j[a] > 0 ? i - st[a] : i, ip = j[a] < n - 1 ? i + st[a] : i;
        const double a0 = p0[im], b0 = p0[ip];
        if (a0 * p0i < 0.0 || b0 * p0i < 0.0) near = true;
        double d = fabs(b0 - a0) / 2.0;
        d = fmax(d, fabs(b0 - p0i));
        d = fmax(d, fabs(p0i - a0));
        dmax = fmax(dmax, d);
        const double bm = (pi - p[im]) / h, fw = (p[ip] - pi) / h;   // backward, forward
        double u2, v2;
        if (s > 0.0) {
            u2 = bm > 0.0 ? bm * bm : 0.0;
            v2 = fw < 0.0 ? fw * fw : 0.0;
        } else {
            u2 = bm < 0.0 ? bm * bm : 0.0;
            v2 = fw > 0.0 ? fw * fw : 0.0;
        }
        g += u2 > v2 ? u2 : v2;
    }
    if (s == 0.0) q[i] = pi;
    else if (near && dmax > 0.0) q[i] = pi - dt / h * (s * fabs(pi) - h * p0i / dmax);
    else q[i] = pi - dt * s * (sqrt(g) - 1.0);
}

}  // namespace

extern "C" gcmg_status gcmg_reinit(int dim, int n, const double *phi0_dev, int steps, double *phi_dev,
                                   void *stream) {
    if ((dim != 2 && dim != 3) || n < 3 || steps < 0 || !phi0_dev || !phi_dev || phi0_dev == phi_dev)
        return GCMG_E_ARG;
    int64_t nn = 1;
    for (int a = 0; a < dim; a++) nn *= n;
    cudaStream_t s = (cudaStream_t)stream;
    double *tmp = nullptr;
    if (steps > 0 && cudaMalloc(&tmp, nn * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return GCMG_E_OOM;
    }
    cudaError_t e = cudaMemcpyAsync(phi_dev, phi0_dev, nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    const unsigned blocks = (unsigned)((nn + 255) / 256);
    double *a = phi_dev, *b = tmp;
    for (int k = 0; k < steps && e == cudaSuccess; k++) {
        if (dim == 2) k_reinit_step<2><<<blocks, 256, 0, s>>>(n, nn, phi0_dev, a, b);
        else k_reinit_step<3><<<blocks, 256, 0, s>>>(n, nn, phi0_dev, a, b);
        e = cudaGetLastError();
        double *t = a;
        a = b;
        b = t;
    }
    if (e == cudaSuccess && a != phi_dev)
        e = cudaMemcpyAsync(phi_dev, a, nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (tmp) cudaFree(tmp);
    return e == cudaSuccess ? GCMG_OK : GCMG_E_CUDA;
}
