// FP64-accuracy weighted sweeps evaluated on the FP32 pipe, in float-float arithmetic.
//
// GB300 issues FP64 fused multiply-adds at ~1/74 of its FP32 rate, so the FP64 sweep (every one
// of its 8 operations per 9-point update an FP64 instruction) is bound by the FP64 pipe at ~0.22
// of the HBM bandwidth.  Here the iterate and b are held as unevaluated pairs of floats, hi + lo
// with |lo| <= ulp(hi)/2 (48 significant bits against FP64's 53), and the sweep
// u' = u + w (L u - b) of Sec. 2.1 is evaluated with the error-free transformations of Knuth
// (TwoSum: s + e = a + b exactly) and Dekker (TwoProduct, here in its fused-multiply-add form:
// p + e = a b exactly).  17 points: in the evaluation order of the FP64 sweep (the shared y-march
// of stencil_dev.cuh, with float-float in place of double).  5 and 9 points: a y-march of its own,
// with the next row's loads issued ahead, in the algebraically equal scaled form
//   u' = (1 - c w / D) u + (w / D) (S - D b),
// S the neighbour sum of D L u + c u with coefficients 1 and 4 (D = 1, c = 4 for 5 points; D = 6,
// c = 20 for 9 points, Eq. 1 times 6): S needs float-float adds and one exact scaling by 4, D b is
// formed once when b is converted, and w / D and 1 - c w / D are rounded once per sweep on the host
// -- 69 and 93 FP32 operations per update against 80 and 116 for the three float-float
// multiply-adds of the FP64 sweep's form.  The pair occupies the same 8 bytes as a double,
// so the sweep moves the FP64 sweep's bytes with FP32 instructions only.  The result is not the
// FP64 sweep's bits: it agrees with it to a few units of 2^-47 of the terms it adds (in the scaled
// form, |c1 u| and |w / D| |S - D b|, each at most about 3.4 |w| max|u| + |w| max|b| for 9 points), well
// inside the per-sweep tolerance of 1e-12 x (max|u| + |w| (9 max|u| + max|b|)) the sweeps are held to.
//
// Conversions: the plan's padded FP64 buffers are converted in place to float-float before the
// sweeps (hi = fl32(d), lo = fl32(d - hi)) and back after them (fl64(hi + lo)); values must lie in
// the float range (|d| < 3.4e38); below 2^-126 their low part is lost (relative error 2^-24 of a
// value that small).  Homogeneous-Dirichlet plans only: their ghost ring is 0 or the reflection of
// the interior, which the sweeps rewrite, so no boundary data passes through the conversions.
#include "cj_internal.h"
#include "grid_dev.cuh"
#include "stencil_dev.cuh"

namespace {

struct __align__(8) ff {
    float hi, lo;
};

__device__ __forceinline__ ff operator-(ff a) { return ff{-a.hi, -a.lo}; }

// Knuth's TwoSum: s + e = a + b exactly (6 operations, no condition on |a|, |b|).
__device__ __forceinline__ ff two_sum_f(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return ff{s, e};
}

// Dekker's FastTwoSum: s + e = a + b exactly when |a| >= |b| (or a = 0).
__device__ __forceinline__ ff fast_two_sum_f(float a, float b) {
    const float s = a + b;
    return ff{s, b - (s - a)};
}

// a + b: TwoSum of the high parts, the low parts added to its error, renormalised; the error is a
// few units of 2^-47 of |a| + |b|.
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum_f(a.hi, b.hi);
    return fast_two_sum_f(s.hi, s.lo + (a.lo + b.lo));
}

// a * b: the exact product of the high parts by a fused multiply-add (TwoProduct), the cross
// terms added to its error, renormalised.
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum_f(p, e);
}

// a - b
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, -b); }

// a times a power of two (exact: both parts scale without rounding)
__device__ __forceinline__ ff ff_scale2(ff a, float two_k) { return ff{a.hi * two_k, a.lo * two_k}; }

// float-float of a double, rounded once per part (host and device)
__host__ __device__ __forceinline__ ff ff_of(double d) {
    const float hi = (float)d;
    return ff{hi, (float)(d - (double)hi)};
}

}  // namespace

namespace {

template <>
struct Ar<ff> {
    static __device__ __forceinline__ ff add(ff a, ff b, ff) { return ff_add(a, b); }
    static __device__ __forceinline__ ff fm(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }
};

// The stencil coefficients of h^2 Delta_h as float-float (each rounded once from its FP64 value).
template <>
struct Co<ff> {
    static __device__ __forceinline__ ff c5() { return ff{-4.0f, 0.0f}; }
    static __device__ __forceinline__ ff ax9() { return ff_of(4.0 / 6.0); }
    static __device__ __forceinline__ ff dg9() { return ff_of(1.0 / 6.0); }
    static __device__ __forceinline__ ff cc9() { return ff_of(-20.0 / 6.0); }
    static __device__ __forceinline__ ff a1() { return ff_of(64.0 / 72.0); }
    static __device__ __forceinline__ ff a2() { return ff_of(-4.0 / 72.0); }
    static __device__ __forceinline__ ff d1() { return ff_of(16.0 / 72.0); }
    static __device__ __forceinline__ ff d2() { return ff_of(-1.0 / 72.0); }
    static __device__ __forceinline__ ff cc17() { return ff_of(-300.0 / 72.0); }
};

template <>
__device__ __forceinline__ ff ld<ff>(const ff *p) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return ff{v.x, v.y};
}

// The weights of one sweep.  17 points: w, for u' = u + w (L u - b) in the FP64 sweep's order.
// 5 and 9 points, in the scaled form D L u = sum of the neighbours with small integer
// coefficients - c u (D = 1, c = 4; D = 6, c = 20), with b stored as D b:
//   u' = c1 u + wD (D L u + c u - D b),   wD = w / D,   c1 = 1 - c wD,
// so the neighbour sum needs no multiplication (its coefficients 1 and 4 are powers of two).
struct FFWeights {
    ff w, wD, c1;
};

template <int ST>
struct SweepOpFF {
    ff *out;
    const Grid *g;
    int i;
    FFWeights w;
    __device__ __forceinline__ void operator()(int j, ff r, ff uc) {
        store_node<(ST == 17 ? 2 : 1), ff>(out, *g, i, j, Ar<ff>::fm(w.w, r, uc));
    }
    // t = D L u + c u - D b at (i, j): the new value c1 u + wD t
    __device__ __forceinline__ void scaled(int j, ff t, ff uc) {
        store_node<1, ff>(out, *g, i, j, ff_add(ff_mul(w.c1, uc), ff_mul(w.wD, t)));
    }
};

// Blocks of kBX threads resident per SM: 16 (32 registers a thread) for the 5- and 9-point
// sweeps, 10 for the 17-point one, whose five-row window needs about 50.
__host__ __device__ constexpr int ff_blocks_per_sm(int st) { return st == 17 ? 10 : 16; }

// The y-march of the 5- and 9-point sweeps (the FP64 sweep's order), with the loads of row j + 1
// (and b of row j) issued one iteration ahead: each iteration's dependent float-float chain is
// long, so the next row's memory latency is hidden behind it.  Row indices are clamped to the
// strip's last row + 1 (a row every strip has), so the last iteration reloads it harmlessly.
template <int ST>
__device__ __forceinline__ void march_ff(const ff *__restrict__ u, const ff *__restrict__ b, const Grid &g,
                                         int i, int j0, int j1, SweepOpFF<ST> &op) {
    const long long P = g.pitch;
    const ff *col = u + g.idx(i, 0);
    const ff *bcol = b + g.idx(i, 0);
    if (ST == 5) {
        ff um = ld(col + (long long)(j0 - 1) * P);
        ff uc = ld(col + (long long)j0 * P);
        const ff *row = col + (long long)j0 * P;
        ff nu = ld(row + P), nl = ld(row - 1), nr = ld(row + 1), nb = ld(bcol + (long long)j0 * P);
        for (int j = j0; j <= j1; ++j) {
            const ff up = nu, l = nl, r_ = nr, bk = nb;
            const int jn = min(j + 1, j1);
            row = col + (long long)jn * P;
            nu = ld(row + P);
            nl = ld(row - 1);
            nr = ld(row + 1);
            nb = ld(bcol + (long long)jn * P);
            const ff p0 = ff_add(l, r_);
            const ff v1 = ff_add(um, up);
            const ff a = ff_add(p0, v1);
            op.scaled(j, ff_sub(a, bk), uc);
            um = uc;
            uc = up;
        }
    } else {
        const ff *row = col + (long long)(j0 - 1) * P;
        ff um = ld(row);
        ff pm = ff_add(ld(row - 1), ld(row + 1));
        row += P;
        ff uc = ld(row);
        ff pc = ff_add(ld(row - 1), ld(row + 1));
        row += P;
        ff nu = ld(row), nl = ld(row - 1), nr = ld(row + 1), nb = ld(bcol + (long long)j0 * P);
        // unrolled by 2, so the rotation of the window (um, uc, pm, pc and the rows in flight)
        // is register renaming rather than moves: 160 -> 170 Gupd/s on 4096^2
#pragma unroll 2
        for (int j = j0; j <= j1; ++j) {
            const ff up = nu, l = nl, r_ = nr, bk = nb;
            const int jn = min(j + 1, j1);
            row = col + (long long)(jn + 1) * P;
            nu = ld(row);
            nl = ld(row - 1);
            nr = ld(row + 1);
            nb = ld(bcol + (long long)jn * P);
            const ff pp = ff_add(l, r_);
            const ff v1 = ff_add(um, up);
            const ff a = ff_add(pc, v1);
            const ff d = ff_add(pm, pp);
            op.scaled(j, ff_sub(ff_add(ff_scale2(a, 4.0f), d), bk), uc);
            um = uc;
            uc = up;
            pm = pc;
            pc = pp;
        }
    }
}

// One weighted sweep out = u + w (L u - b) in float-float on the padded grids (homogeneous plans:
// the 17-point stencil's reflection ghosts are rewritten with each node).
template <int ST>
__global__ void __launch_bounds__(kBX, ff_blocks_per_sm(ST)) sweep_ff_kernel(const ff *__restrict__ u,
                                                                        const ff *__restrict__ b,
                                                                        ff *__restrict__ out, Grid g, int ty,
                                                                        FFWeights w) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    const int j0 = blockIdx.y * ty + 1;
    const int j1 = min(j0 + ty - 1, g.Ny);
    if (i > g.Nx) return;
    SweepOpFF<ST> op{out, &g, i, w};
    if (ST == 17)
        march<ST, ff>(u, b, g, i, j0, j1, ff{1.0f, 0.0f}, op);
    else
        march_ff<ST>(u, b, g, i, j0, j1, op);
}

// Launch shape: 128-column strips of ty rows, about ff_blocks_per_sm blocks per SM in one wave
// (rows per strip at least 4, 8 for the 17-point stencil, against the rows a strip re-reads).
dim3 ff_grid(const Grid &g, int st, int *ty) {
    const int nbx = (g.Nx + kBX - 1) / kBX;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long nby = (long long)(sms > 0 ? sms : 1) * ff_blocks_per_sm(st) / nbx;
    if (nby < 1) nby = 1;
    if (nby > g.Ny) nby = g.Ny;
    const int min_ty = st == 17 ? 8 : 4;
    int t = (int)((g.Ny + nby - 1) / nby);
    if (t < min_ty) t = min_ty < g.Ny ? min_ty : g.Ny;
    *ty = t;
    return dim3(nbx, (g.Ny + t - 1) / t);
}

// In place: doubles -> float-float pairs of D times them (D = 1 for u; the scale of the sweep's
// form for b), and back (times 1 / D, exact for D = 1; b is imported again by every call that
// uses it, so its value after the sweeps is not read).
__global__ void __launch_bounds__(256) to_ff_kernel(double *a, long long n, double D) {
    for (long long k = blockIdx.x * 256LL + threadIdx.x; k < n; k += (long long)gridDim.x * 256) {
        const ff v = ff_of(D * a[k]);
        reinterpret_cast<ff *>(a)[k] = v;
    }
}

__global__ void __launch_bounds__(256) from_ff_kernel(double *a, long long n, double inv_D) {
    for (long long k = blockIdx.x * 256LL + threadIdx.x; k < n; k += (long long)gridDim.x * 256) {
        const ff v = reinterpret_cast<const ff *>(a)[k];
        a[k] = ((double)v.hi + (double)v.lo) * inv_D;
    }
}

cudaError_t convert(double *a, long long n, bool to_ff, cudaStream_t s, double D = 1.0) {
    const long long blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    if (to_ff)
        to_ff_kernel<<<(int)blocks, 256, 0, s>>>(a, n, D);
    else
        from_ff_kernel<<<(int)blocks, 256, 0, s>>>(a, n, 1.0 / D);
    return cudaGetLastError();
}

// D and c of the scaled form of the 5- and 9-point sweeps (1 for 17 points, which keeps the
// FP64 sweep's form).
double ff_scale(int st) { return st == 9 ? 6.0 : 1.0; }
double ff_centre(int st) { return st == 9 ? 20.0 : 4.0; }

}  // namespace

bool ff_sweeps_supported(const cj_plan *p) {
    return p && p->precision == CJ_FP64 && p->pattern == 0 && p->bc == CJ_BC_DIRICHLET0 && p->u1;
}

cudaError_t launch_sweeps_ff(const cj_plan *p, const double *const *bufs, long long first, long long count,
                             int *cur_out, cudaStream_t s) {
    *cur_out = 0;
    if (count == 0) return cudaSuccess;  // no sweep: the iterate passes through unrounded
    const long long n = p->g64.elems();
    double *u[2] = {const_cast<double *>(bufs[0]), const_cast<double *>(bufs[1])};
    double *b = const_cast<double *>(bufs[2]);
    const double D = ff_scale(p->st);
    cudaError_t e = convert(b, n, true, s, D);
    if (e == cudaSuccess) e = convert(u[0], n, true, s);
    if (e == cudaSuccess) e = convert(u[1], n, true, s);
    int cur = 0, ty = 1;
    const dim3 grid = ff_grid(p->g64, p->st, &ty);
    for (long long k = 0; k < count && e == cudaSuccess; ++k) {
        const double wk = p->w[(first + k) % p->M], wD = wk / D;
        const FFWeights w{ff_of(wk), ff_of(wD), ff_of(1.0 - ff_centre(p->st) * wD)};
        const ff *ui = reinterpret_cast<const ff *>(u[cur]);
        ff *uo = reinterpret_cast<ff *>(u[cur ^ 1]);
        const ff *bb = reinterpret_cast<const ff *>(b);
        switch (p->st) {
            case 5: sweep_ff_kernel<5><<<grid, kBX, 0, s>>>(ui, bb, uo, p->g64, ty, w); break;
            case 9: sweep_ff_kernel<9><<<grid, kBX, 0, s>>>(ui, bb, uo, p->g64, ty, w); break;
            default: sweep_ff_kernel<17><<<grid, kBX, 0, s>>>(ui, bb, uo, p->g64, ty, w); break;
        }
        e = cudaGetLastError();
        cur ^= 1;
    }
    if (e == cudaSuccess) e = convert(u[0], n, false, s);
    if (e == cudaSuccess) e = convert(u[1], n, false, s);
    if (e == cudaSuccess) e = convert(b, n, false, s, D);
    *cur_out = cur;
    return e;
}
