// Host build of the exact Laplacian-numerator sum (csrc/exact_lap.h) for
// tests/test_exact_lap.py: the same header the device kernels include.
#include "exact_lap.h"

extern "C" int exl_lap(int n, double up, const double *nb, double *out) {
    if (n == 4) {
        const double a[4] = {nb[0], nb[1], nb[2], nb[3]};
        return exl::lap_sum_exact<4>(up, a, out) ? 1 : 0;
    }
    if (n == 6) {
        const double a[6] = {nb[0], nb[1], nb[2], nb[3], nb[4], nb[5]};
        return exl::lap_sum_exact<6>(up, a, out) ? 1 : 0;
    }
    return -1;
}
