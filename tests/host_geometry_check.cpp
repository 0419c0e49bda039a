// Test program (built and run by tests/test_host_geometry.py, host only):
// builds the level hierarchy of the 3D torus with the library's own setup
// code and checks the work lists the 3D kernels walk against their
// definitions, printing one line "name failures count" per check.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "gcmg_internal.h"

using namespace gcmg;

static int64_t idx(const HostLevel &L, int i, int j, int k) { return ((int64_t)i * L.n + j) * L.n + k; }
static int kind(const HostLevel &L, int64_t p) { return L.type[p] & NODE_KIND; }

int main(int argc, char **argv) {
    const int n = argc > 1 ? std::atoi(argv[1]) : 65;
    const int mu = 10;
    std::vector<double> phi((size_t)n * n * n);
    const double h = 2.0 / (n - 1);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) {
                const double x = -1 + i * h, y = -1 + j * h, z = -1 + k * h;
                phi[((size_t)i * n + j) * n + k] = std::sqrt(std::pow(std::sqrt(x * x + y * y) - 0.5, 2) + z * z) - 0.25;
            }
    std::vector<HostLevel> H;
    build_hierarchy(3, n, 9, phi.data(), 3.0, H);
    long fails = 0;
    auto report = [&](const char *name, long f, long cnt) {
        std::printf("%s %ld %ld\n", name, f, cnt);
        fails += f;
    };
    for (size_t l = 0; l < H.size(); l++) {
        HostLevel &L = H[l];
        const int ln = L.n;
        // row segments: every inside node in exactly one segment of at most
        // 64 consecutive inside nodes of one row
        {
            std::vector<int> hit(L.nn, 0);
            long f = 0, cnt = 0;
            for (size_t s = 0; s < L.sp_list.size(); s += 2) {
                const int64_t r = L.sp_list[s];
                const uint32_t w = (uint32_t)L.sp_list[s + 1];
                const int k0 = (int)(w & 0xffffu), k1 = (int)(w >> 16);
                if (k1 < k0 || k1 - k0 + 1 > 64 || k1 >= ln) f++;
                for (int k = k0; k <= k1 && k < ln; k++) {
                    const int64_t p = r * ln + k;
                    if (kind(L, p) != NODE_IN) f++;
                    hit[p]++;
                }
                cnt++;
            }
            for (int64_t p = 0; p < L.nn; p++)
                if ((kind(L, p) == NODE_IN) != (hit[p] == 1)) f++;
            report("segments", f, cnt);
        }
        // red-sweep sources: node, or -1 - q of the ghost at that neighbour,
        // in the order -1, +1, -s0, +s0, -s1, +s1
        {
            long f = 0;
            const size_t m = L.band_red.size();
            const int64_t off[6] = {-1, 1, -L.stride[0], L.stride[0], -L.stride[1], L.stride[1]};
            for (size_t i = 0; i < m; i++)
                for (int k = 0; k < 6; k++) {
                    const int64_t q = (int64_t)L.band_red[i] + off[k];
                    const int32_t sv = L.band_red_src[(size_t)k * m + i];
                    if (kind(L, q) == NODE_GHOST) {
                        if (sv >= 0 || L.ghost_node[-1 - sv] != q) f++;
                    } else if (sv != q) {
                        f++;
                    }
                }
            report("red_sources", f, (long)m);
        }
        // box stencils: the decoded nodes equal the stored ones
        {
            long f = 0, boxes = 0;
            for (int64_t q = 0; q < L.ng(); q++) {
                const unsigned code = L.gcode[q];
                if (!code) continue;
                boxes++;
                const int mm = (int)(code & 3u);
                const int64_t D0 = (code & 4u) ? -L.stride[0] : L.stride[0], D1 = (code & 8u) ? -L.stride[1] : L.stride[1];
                const int64_t D2 = (code & 16u) ? -1 : 1;
                for (int k = 0; k < KMAX; k++) {
                    int64_t want = L.ghost_node[q];
                    if (mm == 3) want = L.gbase[q] + (k / 9) * D0 + ((k / 3) % 3) * D1 + (k % 3) * D2;
                    else if (k < 8) want = L.gbase[q] + (k / 4) * D0 + ((k / 2) % 2) * D1 + (k % 2) * D2;
                    if (L.stn[q * KMAX + k] != want) f++;
                }
                if (mm == 2)
                    for (int k = 8; k < KMAX; k++)
                        if (L.wD[q * KMAX + k] != 0.0 || L.wN[q * KMAX + k] != 0.0) f++;
            }
            report("box_stencils", f, boxes);
        }
        // partial-transfer list: exactly the coarse inside nodes whose fine
        // 27-neighbourhood is not all inside; FP64 weights equal the
        // independent routine to rounding, FP32 weights are them rounded
        if (l + 1 < H.size()) {
            const HostLevel &C = H[l + 1];
            long f = 0;
            std::vector<int32_t> want;
            for (int i = 0; i < C.n; i++)
                for (int j = 0; j < C.n; j++)
                    for (int k = 0; k < C.n; k++) {
                        const int64_t c = idx(C, i, j, k);
                        if (kind(C, c) != NODE_IN) continue;
                        bool full = true;
                        for (int a = -1; a <= 1; a++)
                            for (int b = -1; b <= 1; b++)
                                for (int d = -1; d <= 1; d++)
                                    if (kind(L, idx(L, 2 * i + a, 2 * j + b, 2 * k + d)) != NODE_IN) full = false;
                        if (!full) want.push_back((int32_t)c);
                    }
            if (want != L.partial_coarse) f++;
            const size_t m = L.partial_coarse.size();
            for (size_t t = 0; t < m && f == 0; t++) {
                const int64_t c = L.partial_coarse[t];
                const int i = (int)(c / C.stride[0]), j = (int)((c / C.stride[1]) % C.n), k = (int)(c % C.n);
                double wt[27];
                const bool any = partial_transfer_weights(L, idx(L, 2 * i, 2 * j, 2 * k), true, wt);
                for (int s = 0; s < 27; s++) {
                    const double wd = L.partial_wd[(size_t)s * m + t];
                    const float wf = L.partial_wf[(size_t)s * m + t];
                    const double ref = any ? wt[s] : 0.0;
                    if (std::fabs(wd - ref) > 1e-15) f++;
                    if (std::fabs((double)wf - ref) > 1e-7) f++;
                }
            }
            report("partial_transfer", f, (long)m);
        }
        // junction blocks (mu sweeps): every zone node written back by one
        // block; each block updates every zone node within 4 mu of its own
        {
            for (int64_t q = 0; q < L.ng(); q++) L.bc[q] = L.B[q * 3 + 2] < 0 ? 1 : 0;
            build_junction(L, 2.0, mu);
            const LocalProgram &P = L.junction;
            long f = 0;
            std::vector<int> wb(L.nn, 0);
            std::vector<uint8_t> zone(L.nn, 0);
            for (int32_t p : P.zred) zone[p] = 1;
            for (int32_t p : P.zblack) zone[p] = 1;
            for (int32_t q : P.zghost) zone[L.ghost_node[q]] = 1;
            for (int c = 0; c < P.ncomp(); c++) {
                const int b0 = P.node_off[c], nw = P.wb_cnt[c];
                std::vector<uint8_t> upd(L.nn, 0);
                // the component's updated nodes: its inside and ghost entries
                for (int e = P.int_off[c]; e < P.int_off[c + 1]; e++) upd[P.int_glob[e]] = 1;
                for (int e = P.gh_off[c]; e < P.gh_off[c + 1]; e++) upd[L.ghost_node[P.gh_q[e]]] = 1;
                for (int e = 0; e < nw; e++) {
                    const int64_t p = P.lnode[b0 + e];
                    wb[p]++;
                    if (!P.blocked) continue;
                    const int pi = (int)(p / L.stride[0]), pj = (int)((p / L.stride[1]) % ln), pk = (int)(p % ln);
                    const int R = 4 * mu;
                    for (int a = std::max(0, pi - R); a <= std::min(ln - 1, pi + R); a++)
                        for (int b = std::max(0, pj - R); b <= std::min(ln - 1, pj + R); b++)
                            for (int d = std::max(0, pk - R); d <= std::min(ln - 1, pk + R); d++) {
                                const int64_t x = idx(L, a, b, d);
                                if (zone[x] && !upd[x]) f++;
                            }
                }
            }
            long zn = 0;
            for (int64_t p = 0; p < L.nn; p++) {
                if (zone[p]) zn++;
                if (zone[p] ? wb[p] != 1 : wb[p] != 0) f++;
            }
            std::printf("junction_blocked %d\n", (int)P.blocked);
            report("junction_blocks", f, zn);
        }
    }
    std::printf("total_failures %ld\n", fails);
    return fails ? 1 : 0;
}
