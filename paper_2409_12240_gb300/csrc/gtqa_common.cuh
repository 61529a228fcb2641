// Small device-side toolkit shared by the GTQA kernels: complex arithmetic,
// thread-team synchronisation, butterfly reductions and the batched one-sided
// Jacobi SVD used for every small matrix decomposition of the method.
#pragma once

#include <climits>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gtqa {

// ---------------------------------------------------------------------------
// complex numbers over float or double
// ---------------------------------------------------------------------------
template <typename R>
struct __align__(sizeof(R) * 2) C {
    R x, y;
};
using cd = C<double>;
using cf = C<float>;

template <typename R> __device__ __forceinline__ C<R> cmk(R a, R b) { return C<R>{a, b}; }
template <typename R> __device__ __forceinline__ C<R> operator+(C<R> a, C<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R> __device__ __forceinline__ C<R> operator-(C<R> a, C<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R> __device__ __forceinline__ C<R> operator*(C<R> a, C<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R> __device__ __forceinline__ C<R> operator*(R s, C<R> a) { return {s * a.x, s * a.y}; }
template <typename R> __device__ __forceinline__ C<R> conj(C<R> a) { return {a.x, -a.y}; }
template <typename R> __device__ __forceinline__ R norm2(C<R> a) { return a.x * a.x + a.y * a.y; }
// acc + a * b
template <typename R> __device__ __forceinline__ C<R> cfma(C<R> a, C<R> b, C<R> acc) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}
// acc + conj(a) * b
template <typename R> __device__ __forceinline__ C<R> cfmac(C<R> a, C<R> b, C<R> acc) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
    return acc;
}
template <typename To, typename From> __device__ __forceinline__ C<To> ccast(C<From> a) {
    return C<To>{(To)a.x, (To)a.y};
}

// ---------------------------------------------------------------------------
// thread groups: G contiguous lanes inside one warp, G a power of two <= 32
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (G >= 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
}

// Butterfly sum over aligned groups of G lanes.  Every lane ends with the same
// bits: at each level a lane adds a + b while its partner adds b + a.
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off);
    return v;
}

// Synchronisation policy for a group that lives inside one warp.
struct WarpGroup {
    unsigned mask;
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    __device__ __forceinline__ bool any(int p) const { return __any_sync(mask, p) != 0; }
    __device__ __forceinline__ int max_int(int v) const { return __reduce_max_sync(mask, v); }
    __device__ __forceinline__ unsigned or_bits(unsigned v) const { return __reduce_or_sync(mask, v); }
};

// Synchronisation policy for a group that is the whole thread block.
struct BlockGroup {
    int* flag;  // one int of shared memory
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ bool any(int p) const {
        __syncthreads();
        if (threadIdx.x == 0) *flag = 0;
        __syncthreads();
        if (p) atomicOr(flag, 1);
        __syncthreads();
        return *flag != 0;
    }
    __device__ __forceinline__ int max_int(int v) const {
        __syncthreads();
        if (threadIdx.x == 0) *flag = INT_MIN;
        __syncthreads();
        atomicMax(flag, v);
        __syncthreads();
        return *flag;
    }
    __device__ __forceinline__ unsigned or_bits(unsigned v) const {
        __syncthreads();
        if (threadIdx.x == 0) *flag = 0;
        __syncthreads();
        if (v) atomicOr(reinterpret_cast<unsigned*>(flag), v);
        __syncthreads();
        return *reinterpret_cast<volatile unsigned*>(flag);
    }
};

// ---------------------------------------------------------------------------
// Reciprocal and (reciprocal) square root without the FP64 divide/sqrt sequences,
// which cost ~10-15 FP64 pipe instructions each on this part.  A hardware seed
// (PTX rcp.approx.ftz.f64 / rsqrt.approx.ftz.f64, ~2^-22 relative error) is refined by
// two Newton-Raphson steps (quadratic convergence: error ~2^-88, i.e. FP64 rounding).
// Float versions use the single-precision hardware approximations directly.
// Inputs must be finite and positive (callers guard zero).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double nr_rcp(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}
// one refinement step only: relative error ~2^-44, for results that are rounded to FP32
__device__ __forceinline__ double nr_rcp1(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return fma(r, fma(-x, r, 1.0), r);
}
__device__ __forceinline__ double nr_rsqrt(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    // y <- y + y (1 - x y^2) / 2
    double e = fma(-x * y, y, 1.0);
    y = fma(0.5 * y, e, y);
    e = fma(-x * y, y, 1.0);
    return fma(0.5 * y, e, y);
}
__device__ __forceinline__ double nr_sqrt(double x) {
    if (!(x > 0.0)) return 0.0;
    const double y = nr_rsqrt(x);
    const double s = x * y;
    return fma(0.5 * y, fma(-s, s, x), s);   // one correction of s = sqrt(x)
}
__device__ __forceinline__ float nr_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ float nr_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ float nr_sqrt(float x) { return x > 0.f ? sqrtf(x) : 0.f; }

// ---------------------------------------------------------------------------
// Batched one-sided (Hestenes) Jacobi SVD of an N x N complex matrix.
//
// A and V are column-major in shared memory (element (row r, col c) at c*N + r).
// The group has N*N/2 threads: thread g works on pair k = g / N at row r = g % N,
// so the N lanes of a pair are contiguous and reduce with shuffles.  Columns are
// paired by the round-robin (circle) ordering, N/2 disjoint pairs per step and
// N-1 steps per sweep.  For a pair (p, q) with alpha = |a_p|^2, beta = |a_q|^2,
// gamma = a_p^H a_q, the 2x2 unitary J = [[c, s e],[-s conj(e), c]] (e = gamma/|gamma|,
// t = tan(theta) the smaller root of t^2 + 2 zeta t - 1 = 0, zeta = (beta-alpha)/(2|gamma|))
// makes the rotated columns orthogonal.  Sweeps stop when no pair has
// |gamma| > tol * sqrt(alpha beta).  On exit A holds U*S (columns unsorted) and
// V the accumulated right rotations: A_in = (A_out) V^H.
// ---------------------------------------------------------------------------
// Zeroes the entries of an N x N complex matrix (column-major, shared) that lie more than 2^100
// (about 1e30) below its largest entry.  Every value kept by the method's cut-offs (singular
// values above 1e-14 s_0, message eigenvalues above 1e-13 w_max) is far above that, while such
// rounding-level columns would keep one-sided Jacobi rotating pairs whose angle underflows
// (a column of norm ~1e-44 next to one of norm ~1 in the early anneal).  The test compares the
// exponent bits of the entries, on the integer pipe.  The group has N^2/2 lanes.
__device__ __forceinline__ int exp_bits(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff); }
template <int N, typename Group>
__device__ void prune_noise(C<double>* A, int g, const Group& grp) {
    constexpr int NN = N * N, L = NN / 2;
    int e = 0;
#pragma unroll
    for (int j = 0; j < NN / L; ++j) {
        const C<double> a = A[g + j * L];
        e = max(e, max(exp_bits(a.x), exp_bits(a.y)));
    }
    const int emax = grp.max_int(e);
#pragma unroll
    for (int j = 0; j < NN / L; ++j) {
        const C<double> a = A[g + j * L];
        if (max(exp_bits(a.x), exp_bits(a.y)) < emax - 100) A[g + j * L] = C<double>{0.0, 0.0};
    }
    grp.sync();
}

__device__ __forceinline__ void round_robin_pair(int N, int step, int k, int& p, int& q) {
    if (k == 0) {
        p = step;
        q = N - 1;
    } else {
        p = (step + k) % (N - 1);
        q = (step - k + (N - 1)) % (N - 1);
    }
    if (p > q) { int t = p; p = q; q = t; }
}

// Options: WITHV = false skips the V updates (only the singular values are wanted).
// F32ANGLE (R = double): the rotation angle t is solved in FP32 from the FP64 zeta, and c,
// s and the phase e are then formed in FP64 from that t, so every rotation is unitary to
// FP64 rounding and the FP64 orthogonality test decides convergence; only the size of
// each step is FP32-accurate.  quad_tol > 0: a sweep whose examined pairs all have
// |gamma| <= quad_tol sqrt(alpha beta) is the last one: with quadratic convergence the
// next sweep would find |gamma| ~ quad_tol^2 sqrt(alpha beta) <= tol sqrt(alpha beta) (for
// quad_tol^2 <= tol), so the confirming sweep is skipped.
template <int N, typename R, typename Group, bool WITHV = true, bool F32ANGLE = false>
__device__ int jacobi_svd(C<R>* A, C<R>* V, int g, const Group& grp, unsigned pair_mask,
                          R tol, int max_sweeps, bool init_v, int* nrot = nullptr, R quad_tol = (R)0) {
    const int k = g / N;
    const int r = g % N;
    if (WITHV && init_v) {
        V[(2 * k) * N + r] = C<R>{(R)((2 * k) == r), (R)0};
        V[(2 * k + 1) * N + r] = C<R>{(R)((2 * k + 1) == r), (R)0};
    }
    grp.sync();
    const R tol2 = tol * tol, quad2 = quad_tol * quad_tol;
    // a pair whose |gamma|^2 lies near the bottom of the range is orthogonal in absolute terms
    // (the matrices here are normalised); taking it as converged also keeps the reciprocal
    // square root away from subnormal inputs
    const R gmin = sizeof(R) == 8 ? (R)1e-290 : (R)1e-36;
    const bool quad = quad_tol > (R)0;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        int rotated = 0, big = 0;
        for (int step = 0; step < N - 1; ++step) {
            int p, q;
            round_robin_pair(N, step, k, p, q);
            C<R> ap = A[p * N + r], aq = A[q * N + r];
            R alpha = norm2(ap), beta = norm2(aq);
            C<R> gam = cfmac(ap, aq, C<R>{(R)0, (R)0});
            alpha = group_sum<N>(alpha, pair_mask);
            beta = group_sum<N>(beta, pair_mask);
            gam.x = group_sum<N>(gam.x, pair_mask);
            gam.y = group_sum<N>(gam.y, pair_mask);
            const R g2 = gam.x * gam.x + gam.y * gam.y;
            const R ab = alpha * beta;
            if (g2 > gmin && g2 > tol2 * ab) {
                if (g2 > quad2 * ab) big = 1;
                const R rg = nr_rsqrt(g2);                      // 1 / |gamma|
                const R zeta = (beta - alpha) * ((R)0.5 * rg);
                R t;
                if constexpr (F32ANGLE) {
                    // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) in FP32; for huge zeta (beyond the FP32
                    // range when a column is tiny) t = 1/(2 zeta) in FP64, so the rotation does not vanish
                    const R az = fabs(zeta);
                    if (az < (R)1e18) {
                        const float azf = (float)az;
                        const float tf = __frcp_rn(azf + sqrtf(fmaf(azf, azf, 1.f)));
                        t = (R)(zeta >= (R)0 ? tf : -tf);
                    } else {
                        t = (zeta >= (R)0 ? (R)0.5 : (R)-0.5) * nr_rcp(az);
                    }
                } else {
                    const R az = fabs(zeta);
                    // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), the smaller root; 1/(2 zeta) for huge zeta
                    t = (zeta >= (R)0 ? (R)1 : (R)-1) *
                        (az < (R)1e15 ? nr_rcp(az + nr_sqrt((R)1 + az * az)) : (R)0.5 * nr_rcp(az));
                }
                const R c = nr_rsqrt((R)1 + t * t);
                const R s = c * t;
                const C<R> e = C<R>{gam.x * rg, gam.y * rg};
                const C<R> se = s * e;
                const C<R> sec = conj(se);
                A[p * N + r] = c * ap - sec * aq;
                A[q * N + r] = se * ap + c * aq;
                if constexpr (WITHV) {
                    const C<R> vp = V[p * N + r], vq = V[q * N + r];
                    V[p * N + r] = c * vp - sec * vq;
                    V[q * N + r] = se * vp + c * vq;
                }
                rotated = 1;
                if (nrot && r == 0) ++*nrot;
            }
            grp.sync();
        }
        if (!grp.any(quad ? big : rotated)) {
            ++sweep;
            break;
        }
    }
    return sweep;   // sweeps run, including the final one (without rotations unless quad_tol stopped it)
}

// True if x (an updated squared norm) is negative, zero or below about half of ref, from the
// raw bits only.
__device__ __forceinline__ bool norm_collapsed(double x, double ref) {
    const long long b = __double_as_longlong(x);
    return b <= 0 || (int)((b >> 52) & 0x7ff) + 1 < exp_bits(ref);
}

// FP64 polish of a one-sided Jacobi SVD (same layout, pairing and rotations as
// jacobi_svd<N, double>) for columns that are already nearly orthogonal, as after an
// FP32 solve and an FP64 Newton-Schulz step.  Fewer FP64 instructions per step:
//  * the squared column norms are kept in nrm[N] (shared) and, in steps whose rotations are all
//    small, updated as alpha' = alpha - tau |gamma|^2 and beta' = beta + tau |gamma|^2 (the two
//    eigenvalues of the pair's 2x2 Gram matrix) instead of two reductions per step; after a
//    large rotation, or where the update would remove more than half of a norm (it then
//    cancels), they are recomputed;
//  * the rotation is parametrised by tau = t / |gamma| = 2 sign(D) / (|D| + sqrt(D^2 + 4|gamma|^2)),
//    D = beta - alpha, solved in FP32 on values scaled by an approximate 1/(alpha + beta);
//    then t^2 = tau^2 |gamma|^2, c = 1/sqrt(1 + t^2) and s e = c tau gamma are formed in FP64,
//    so c^2 + |s e|^2 = 1 to FP64 rounding whatever the error of tau, and the FP64
//    orthogonality test alone decides convergence;
//  * c = 1 - t^2/2 + 3t^4/8 when every pair of the group has t^2 < 1e-6 (the dropped terms are
//    below 3.2e-19).
// The quadratic stop of jacobi_svd applies (quad_tol).
// keep_rank < N (the caller keeps at most keep_rank singular triplets, as in the truncation of
// App. D): only pairs that touch a column among the keep_rank largest (with a margin: norms
// within a factor 4 of the keep_rank-th largest at entry count) decide the quadratic stop, and
// a pair of such a column p with a smaller one q is judged by |gamma| against alpha_p (the
// size of the rotation of the kept column) rather than sqrt(alpha_p beta_q).  The kept
// columns then converge as with keep_rank = N, while rotations among discarded columns, which
// leave the kept subspace unchanged, no longer force a confirming sweep.
// PARTIAL: every pair is rotated in the first sweep; a later sweep runs only the steps of the
// round-robin schedule in which the previous sweep made a rotation above quad_tol.  A pair
// whose rotation in a sweep stayed below quad_tol is orthogonal after it to about quad_tol
// times the largest rotation of that sweep (the rotations of its columns with the others
// reintroduce only products of their sizes), which is the accuracy of the quadratic stop, so
// those steps need no second pass.  Otherwise every pair is rotated in each sweep that runs.
// Returns the sweeps run (partial ones included); *nsteps (if given, group lane 0) counts the
// steps run, of N / 2 pairs each.
template <int N, typename Group, bool PARTIAL = false>
__device__ int jacobi_polish(C<double>* A, C<double>* V, double* nrm, int g, const Group& grp, unsigned pair_mask,
                             double tol, double quad_tol, int max_sweeps, int* nrot, int keep_rank = N,
                             unsigned* relmask = nullptr, int* nsteps = nullptr) {
    using CD = C<double>;
    const int k = g / N;
    const int r = g % N;
    {
        const double n0 = group_sum<N>(norm2(A[(2 * k) * N + r]), pair_mask);
        const double n1 = group_sum<N>(norm2(A[(2 * k + 1) * N + r]), pair_mask);
        if (r == 0) {
            nrm[2 * k] = n0;
            nrm[2 * k + 1] = n1;
        }
    }
    grp.sync();
    const bool partial = keep_rank < N && relmask != nullptr;
    if (partial) {
        if (g == 0) *relmask = 0u;
        grp.sync();
        if (g < N) {
            // the keep_rank-th largest norm, then every column within a factor 4 of it
            const double x = nrm[g];
            int above = 0;
            for (int j = 0; j < N; ++j) above += (nrm[j] > x) || (nrm[j] == x && j < g);
            if (above == keep_rank - 1) {
                const double thr = 0.25 * x;
                unsigned mask = 0u;
                for (int j = 0; j < N; ++j) mask |= (nrm[j] >= thr) ? (1u << j) : 0u;
                *relmask = mask;
            }
        }
        grp.sync();
    }
    const unsigned rel = partial ? *relmask : 0xffffffffu;
    const double tol2 = tol * tol, quad2 = quad_tol * quad_tol;
    static_assert(N - 1 <= 32, "one bit per step");
    unsigned steps = N - 1 == 32 ? 0xffffffffu : (1u << (N - 1)) - 1u;   // steps this sweep runs
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        int big = 0;
        unsigned bigsteps = 0u;   // this lane's steps with a rotation above quad_tol
        for (int step = 0; step < N - 1; ++step) {
            if (PARTIAL && !((steps >> step) & 1u)) continue;   // the same for the whole group
            int bstep = 0;   // this lane's pair rotated by more than quad_tol
            if (nsteps && g == 0) ++*nsteps;
            int p, q;
            round_robin_pair(N, step, k, p, q);
            const CD ap = A[p * N + r], aq = A[q * N + r];
            const double alpha = nrm[p], beta = nrm[q];
            CD gam = cfmac(ap, aq, CD{0.0, 0.0});
            gam.x = group_sum<N>(gam.x, pair_mask);
            gam.y = group_sum<N>(gam.y, pair_mask);
            const double g2 = gam.x * gam.x + gam.y * gam.y;
            const double ab = alpha * beta;
            const bool rot = g2 > 1e-290 && g2 > tol2 * ab;   // as in jacobi_svd
            double tau = 0.0, t2 = 0.0;
            if (rot) {
                const bool rp = (rel >> p) & 1u, rq = (rel >> q) & 1u;
                if (rp && rq) {
                    if (g2 > quad2 * ab) bstep = 1;
                } else if (rp || rq) {
                    const double mx = alpha > beta ? alpha : beta;
                    if (g2 > quad2 * mx * mx) bstep = 1;
                }
                const double d = beta - alpha;
                double rsc;
                asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(rsc) : "d"(alpha + beta));
                const float dn = (float)(d * rsc), gn = (float)(g2 * rsc * rsc);
                const float tn = 2.f * __frcp_rn(fabsf(dn) + sqrtf(fmaf(dn, dn, 4.f * gn)));
                tau = (double)(dn >= 0.f ? tn : -tn) * rsc;
                t2 = tau * tau * g2;
            }
            const bool series = !grp.any(rot && !(t2 < 1e-6));
            if (rot) {
                const double c = series ? fma(t2, fma(0.375, t2, -0.5), 1.0) : nr_rsqrt(1.0 + t2);
                const double ct = c * tau;
                const CD se = CD{ct * gam.x, ct * gam.y};
                const CD sec = conj(se);
                A[p * N + r] = c * ap - sec * aq;
                A[q * N + r] = se * ap + c * aq;
                const CD vp = V[p * N + r], vq = V[q * N + r];
                V[p * N + r] = c * vp - sec * vq;
                V[q * N + r] = se * vp + c * vq;
                if (r == 0 && nrot) ++*nrot;
            }
            // the updated norms; the smaller one loses |m|, and where that cancels (a column nearly
            // parallel to a larger one) the update loses its precision and can turn negative, so
            // both are then recomputed from the columns, as after a large rotation.  The test
            // reads the sign and exponent bits (integer pipe): a drop below half or a sign change
            const double m = tau * g2;   // 0 without a rotation
            const double np_ = alpha - m, nq_ = beta + m;
            const bool exact = !series || (rot && (norm_collapsed(np_, alpha) || norm_collapsed(nq_, beta)));
            if (!exact) {
                if (rot && r == 0) {
                    nrm[p] = np_;
                    nrm[q] = nq_;
                }
            } else {
                // a large rotation: the update alpha - tau |gamma|^2 can cancel, so the two
                // norms are recomputed from the rotated columns
                const double np = group_sum<N>(norm2(A[p * N + r]), pair_mask);
                const double nq = group_sum<N>(norm2(A[q * N + r]), pair_mask);
                if (r == 0) {
                    nrm[p] = np;
                    nrm[q] = nq;
                }
            }
            big |= bstep;
            if (bstep) bigsteps |= 1u << step;
            grp.sync();
        }
        if constexpr (PARTIAL) {
            steps = grp.or_bits(bigsteps);
            if (!steps) {
                ++sweep;
                break;
            }
        } else if (!grp.any(big)) {
            ++sweep;
            break;
        }
    }
    return sweep;
}

// FP64 SVD of an N x N complex matrix A (column-major, shared memory) by the mixed path:
// one-sided Jacobi sweeps on an FP32 copy give V32; one FP64 Newton-Schulz step
// V <- V (3I - V^H V)/2 makes V unitary to ~1e-14; W = A V (FP64) then goes through the
// FP64 polish (jacobi_polish) to orthogonality `tol`.  On exit A holds U S (columns unsorted)
// and V the right singular vectors, as after jacobi_svd<N, double>.  A32, V32 (N^2 complex
// floats), T1, T2 (N^2 complex) and nrm (N) are scratch.  The group has N^2/2 lanes.
template <int N, typename Group>
__device__ int mixed_svd(C<double>* A, C<double>* V, C<float>* A32, C<float>* V32, C<double>* T1, C<double>* T2,
                         double* nrm, int g, const Group& grp, unsigned pair_mask, double tol, double quad_tol,
                         int* nrot, int* sweeps32 = nullptr) {
    using CD = C<double>;
    constexpr int NN = N * N, L = NN / 2;
    for (int t = g; t < NN; t += L) A32[t] = ccast<float>(A[t]);
    grp.sync();
    const int sw32 = jacobi_svd<N, float>(A32, V32, g, grp, pair_mask, 1e-6f, 40, true, nullptr, 1e-3f);
    if (sweeps32) *sweeps32 = sw32;
    for (int t = g; t < NN; t += L) V[t] = ccast<double>(V32[t]);
    grp.sync();
    for (int t = g; t < NN; t += L) {   // T1 = V^H V
        const int q = t / N, p = t % N;
        CD acc = CD{0.0, 0.0};
        for (int r = 0; r < N; ++r) acc = cfmac(V[p * N + r], V[q * N + r], acc);
        T1[t] = acc;
    }
    grp.sync();
    for (int t = g; t < NN; t += L) {   // T2 = V (1.5 I - 0.5 T1)
        const int q = t / N, r = t % N;
        CD acc = 1.5 * V[q * N + r];
        for (int p = 0; p < N; ++p) acc = cfma(-0.5 * V[p * N + r], T1[q * N + p], acc);
        T2[t] = acc;
    }
    grp.sync();
    for (int t = g; t < NN; t += L) {   // T1 = A T2
        const int q = t / N, r = t % N;
        CD acc = CD{0.0, 0.0};
        for (int p = 0; p < N; ++p) acc = cfma(A[p * N + r], T2[q * N + p], acc);
        T1[t] = acc;
    }
    grp.sync();
    for (int t = g; t < NN; t += L) {
        A[t] = T1[t];
        V[t] = T2[t];
    }
    grp.sync();
    return jacobi_polish<N, Group>(A, V, nrm, g, grp, pair_mask, tol, quad_tol, 60, nrot);
}

// Rank of value i among n values, descending, ties by index (used to sort
// singular values without data movement).  A NaN ranks below every number, so the
// ranks are a permutation of 0..n-1 whatever the values.
template <typename R>
__device__ __forceinline__ int desc_rank(const R* v, int n, int i) {
    const R x0 = v[i];
    const R x = (x0 == x0) ? x0 : (R)-INFINITY;
    int rk = 0;
    for (int j = 0; j < n; ++j) {
        const R y0 = v[j];
        const R y = (y0 == y0) ? y0 : (R)-INFINITY;
        rk += (y > x) || (y == x && j < i);
    }
    return rk;
}

}  // namespace gtqa

namespace gtqa {

// ---------------------------------------------------------------------------
// Teams of TEAM threads inside a block: TEAM <= 32 lives in one warp (warp-level
// sync with the team's lane mask); TEAM a multiple of 32 syncs with named barrier
// 1 + team id (barrier 0 stays free for __syncthreads).
// ---------------------------------------------------------------------------
template <int TEAM>
__device__ __forceinline__ void team_bar(int team) {
    if constexpr (TEAM <= 32) {
        __syncwarp(group_mask<TEAM>());
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(TEAM) : "memory");
    }
}

// Synchronisation policy for a multi-warp team (named barrier + shared flag).
template <int TEAM>
struct TeamGroup {
    int team;
    int* flag;
    __device__ __forceinline__ void sync() const { team_bar<TEAM>(team); }
    __device__ __forceinline__ bool any(int p) const {
        team_bar<TEAM>(team);
        if ((threadIdx.x % TEAM) == 0) *flag = 0;
        team_bar<TEAM>(team);
        if (p) atomicOr(flag, 1);
        team_bar<TEAM>(team);
        return *(volatile int*)flag != 0;
    }
    __device__ __forceinline__ int max_int(int v) const {
        team_bar<TEAM>(team);
        if ((threadIdx.x % TEAM) == 0) *flag = INT_MIN;
        team_bar<TEAM>(team);
        atomicMax(flag, v);
        team_bar<TEAM>(team);
        return *(volatile int*)flag;
    }
    __device__ __forceinline__ unsigned or_bits(unsigned v) const {
        team_bar<TEAM>(team);
        if ((threadIdx.x % TEAM) == 0) *flag = 0;
        team_bar<TEAM>(team);
        if (v) atomicOr(reinterpret_cast<unsigned*>(flag), v);
        team_bar<TEAM>(team);
        return *reinterpret_cast<volatile unsigned*>(flag);
    }
};

// L2-coherent loads for data written by other blocks during the same launch.
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ C<double> ldcg(const C<double>* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return C<double>{v.x, v.y};
}
template <>
__device__ __forceinline__ C<float> ldcg(const C<float>* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return C<float>{v.x, v.y};
}

// ---------------------------------------------------------------------------
// Grid-wide barrier for a cooperative (co-resident) launch.  Sense reversal on a
// generation counter; the wait is bounded: after `limit` polls the block records
// GTQA timeout in *err and leaves.  Callers test *err after every barrier and
// return, so a lost block can never hang the device.
// ---------------------------------------------------------------------------
// Grid barrier for cooperative launches over a monotonic 64-bit arrival counter: the
// k-th barrier of a launch completes when the counter reaches base + k * nblocks, so
// an arrival is one release-atomic and the wait one acquire-load poll, with no
// separate generation word to publish.  Thread 0 of each block keeps the target.  Every
// wait is bounded: after `limit` polls the block records GTQA_ERR_TIMEOUT in *err and
// leaves (the others then time out at this or their next barrier).  Launches must pass
// the same number of barriers in every block, which keeps the counter at a multiple of
// nblocks between launches.
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long atom_add_release_u64(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

struct GridBarrier {
    unsigned long long* count;
    int* err;
    unsigned long long next;   // thread 0: counter value that completes the next barrier
    unsigned int nblocks;
};

__device__ __forceinline__ GridBarrier grid_barrier_init(unsigned long long* count, int* err, unsigned int nblocks) {
    GridBarrier gb{count, err, 0ull, nblocks};
    if (threadIdx.x == 0) {
        // at most nblocks - 1 blocks can have arrived at this launch's first barrier
        const unsigned long long c = *(volatile unsigned long long*)count;
        gb.next = c - c % nblocks + nblocks;
    }
    return gb;
}

__device__ __forceinline__ bool grid_sync(GridBarrier& gb, long long limit) {
    __shared__ int ok_shared;
    __syncthreads();   // the block's writes happen before thread 0's release
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long old = atom_add_release_u64(gb.count, 1ull);
        if (old + 1ull < gb.next) {
            long long polls = 0;
            while (ld_acquire_u64(gb.count) < gb.next) {
                if (++polls > limit) {
                    atomicExch(gb.err, 6);   // GTQA_ERR_TIMEOUT
                    ok = 0;
                    break;
                }
                if (polls > 2048) __nanosleep(32);
            }
        }
        gb.next += gb.nblocks;
        ok_shared = ok;
    }
    __syncthreads();
    return ok_shared != 0;   // one value per block, so the whole block leaves together
}

// grid_sync with a step of the first warp between the block's barrier and its arrival: pre()
// runs on warp 0 once the block's shared-memory writes are visible to it, and thread 0's
// release arrival follows in program order, so what pre() writes to global memory is visible
// to every block that passes this barrier.
template <class Pre>
__device__ __forceinline__ bool grid_sync_pre(GridBarrier& gb, long long limit, Pre&& pre) {
    __shared__ int ok_pre;
    __syncthreads();
    if (threadIdx.x < 32) {
        pre();
        __syncwarp();
    }
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long old = atom_add_release_u64(gb.count, 1ull);
        if (old + 1ull < gb.next) {
            long long polls = 0;
            while (ld_acquire_u64(gb.count) < gb.next) {
                if (++polls > limit) {
                    atomicExch(gb.err, 6);   // GTQA_ERR_TIMEOUT
                    ok = 0;
                    break;
                }
                if (polls > 2048) __nanosleep(32);
            }
        }
        gb.next += gb.nblocks;
        ok_pre = ok;
    }
    __syncthreads();
    return ok_pre != 0;
}

// The dynamic shared-memory limit is an attribute of the kernel function, shared by
// every state in the process, while the BP kernel's need grows with the number of
// instances.  The limit is therefore raised to the device maximum (not to one state's
// need), so that states of different sizes can launch the same kernel in any order.
template <class K>
inline cudaError_t raise_smem_limit(K kernel, size_t smem) {
    int dev = 0, mx = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const size_t avail = (size_t)mx > fa.sharedSizeBytes ? (size_t)mx - fa.sharedSizeBytes : 0;
    if (smem > avail) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)avail);
}

}  // namespace gtqa
