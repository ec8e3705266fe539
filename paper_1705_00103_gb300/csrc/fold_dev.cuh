// The odd extension of a grid function with homogeneous Dirichlet data: nodes 0 and N+1
// are zero and the values continue past them as u(-k) = -u(k), u(N+1+k) = -u(N+1-k),
// periodically with period 2(N+1).  The temporal-blocking kernels compute every stage on
// this extension: each operation of the sweep is an odd function of its inputs under
// round-to-nearest, so values on reflected nodes stay the exact negatives of their mirrors
// and interior values equal those of one-sweep launches bit for bit.
#pragma once

namespace {

// Index and sign of node k of the odd extension of 1..N (nodes 0 and N+1 are zero: sign 0).
__device__ __forceinline__ int fold(int k, int N, float &sign) {
    if (k >= 1 && k <= N) {
        sign = 1.0f;
        return k;
    }
    const int P = 2 * (N + 1);
    int m = k % P;
    if (m < 0) m += P;
    if (m == 0 || m == N + 1) {
        sign = 0.0f;
        return 1;
    }
    if (m <= N) {
        sign = 1.0f;
        return m;
    }
    sign = -1.0f;
    return P - m;
}

}  // namespace
