// Per-path device routines shared by the per-bucket kernels and the batched
// persistent kernel.  Lane = sample; all path records are warp-uniform.
#pragma once

#include <type_traits>

#include "qts_device.cuh"

namespace qts {

// How a path adds its phi contributions to the shared tile.
enum PhiMode : int { kPhiNone = 0, kPhiAtomic = 1, kPhiPrivate = 2 };

template <int MODE>
__device__ __forceinline__ void phi_add(float* ps, int idx, float v) {
    if constexpr (MODE == kPhiAtomic) atomicAdd(&ps[idx], v);
    else if constexpr (MODE == kPhiPrivate) ps[idx] += v;  // tile owned by this warp
}

// Per-lane reads of one sample's values by feature index.
struct SmemCols {  // transposed shared tile [feature][kTileLd]; column = lane
    const float* t;
    int lane;
    __device__ __forceinline__ float operator()(int f) const { return t[f * kTileLd + lane]; }
};
struct GlobalCols {  // transposed global copy [feature][ld]; this lane's sample = s
    const float* t;
    int64_t ld;
    int64_t s;
    __device__ __forceinline__ float operator()(int f) const { return __ldg(t + (int64_t)f * ld + s); }
};

// The two extra sums of a pair path's adjoint.  With Q = acc2 - g acc1 the
// pair element's z-gradient at val = 1 and K = acc3 - acc2 + g acc1 (acc3 =
// sum_m w_m U_m, the part of acc2 without the (1 - t_m) factor), per sample
// dL/dval_A = z_A Q + o_A K and dL/dval_B = z_B Q + o_B K; the epilogue adds
// z_k * (sum of Q) from the element's slot, the kernel sums o_A K and o_B K.

// ====================================================== first order ======
//
// c_i = sum_m w_m val prod_{j<i} a_j(t_m) prod_{j>i} a_j(t_m), a_j(t) = z_j + t (o_j - z_j),
// by a prefix product seeded with w_m val and a suffix product (no division),
// two quadrature nodes per f32x2 register pair; phi[f_i] += (o_i - z_i) c_i
// (Thm 1 with S = {i}, Eq. shap_as_weighted_banzhafs).


template <int D, int NP, bool HAS_NAN, typename XR, int PHI = kPhiAtomic, bool PAIRS = false>
__device__ __forceinline__ void fwd_path_f32(const Rec32* __restrict__ r, const XR& xr, float* ps, int lane,
                                             const QuadF& q) {
    constexpr int K = NP / 2;  // node pairs per pass
    const float val = r[0].z;
    const bool pair = PAIRS && (r[D].bits & kPairElem) != 0;
    float dd[D], zz[D];
    int ff[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Rec32 e = r[1 + j];
        const int f = feat_of(e.bits);
        const float x = xr(f);
        const bool o = satisfies<HAS_NAN>(x, e.lo, e.hi, e.bits);
        dd[j] = (o ? 1.f : 0.f) - e.z;
        if (j == D - 1 && pair) dd[j] = pair_d(x, e, r[0]);
        zz[j] = e.z;
        ff[j] = f;
    }
    float cacc[D];
#pragma unroll
    for (int j = 0; j < D; ++j) cacc[j] = 0.f;
    const int npass = q.n_pad / NP;
    for (int pass = 0; pass < npass; ++pass) {
        float2 T[K], P[D][K], A[D][K], S[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int m = pass * NP + 2 * k;
            T[k] = f2(q.t[m], q.t[m + 1]);
            P[0][k] = f2(q.w[m] * val, q.w[m + 1] * val);
        }
        // prefix products P_j = w val prod_{l<j} a_l
#pragma unroll
        for (int j = 0; j < D; ++j) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                A[j][k] = fma2(T[k], f2s(dd[j]), f2s(zz[j]));
                if (j + 1 < D) P[j + 1][k] = mul2(P[j][k], A[j][k]);
            }
        }
        // suffix products, combined on the way down
#pragma unroll
        for (int k = 0; k < K; ++k) S[k] = f2s(1.f);
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            float2 acc = mul2(P[j][0], S[0]);
#pragma unroll
            for (int k = 1; k < K; ++k) acc = fma2(P[j][k], S[k], acc);
            if (j > 0) {
#pragma unroll
                for (int k = 0; k < K; ++k) S[k] = mul2(S[k], A[j][k]);
            }
            cacc[j] += acc.x + acc.y;
        }
    }
#pragma unroll
    for (int j = 0; j < D; ++j) phi_add<PHI>(ps, ff[j] * kTileLd + lane, dd[j] * cacc[j]);
}


// ps: the block's FP64 accumulator tile [feature][kTileLd] (column = lane), or,
// with global_F = F > 0 (the tile does not fit shared memory), this lane's row
// of the FP64 output itself; lanes past the last sample pass live = false.
template <int D, bool HAS_NAN>
__device__ __forceinline__ void fwd_path_f64(const Rec64* __restrict__ r, const float* __restrict__ xs,
                                             double* ps, int lane, const QuadD& q, int global_F = 0,
                                             bool live = true) {
    const double val = r[0].z;
    double dd[D], zz[D], cacc[D];
    int ff[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Rec64 e = r[1 + j];
        const int f = feat_of(e.bits);
        const float x = xs[f * kTileLd + lane];
        const bool o = satisfies<HAS_NAN>(x, e.lo, e.hi, e.bits);
        dd[j] = (o ? 1.0 : 0.0) - e.z;
        zz[j] = e.z;
        ff[j] = f;
        cacc[j] = 0.0;
    }
    for (int m = 0; m < q.n; ++m) {
        const double t = q.t[m];
        double A[D], P[D];
        P[0] = q.w[m] * val;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            A[j] = fma(t, dd[j], zz[j]);
            if (j + 1 < D) P[j + 1] = P[j] * A[j];
        }
        double S = 1.0;
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            cacc[j] += P[j] * S;
            S *= A[j];
        }
    }
    if (!live) return;
    if (global_F == 0) {
#pragma unroll
        for (int j = 0; j < D; ++j) atomicAdd(&ps[ff[j] * kTileLd + lane], dd[j] * cacc[j]);
    } else {
#pragma unroll
        for (int j = 0; j < D; ++j)
            if (ff[j] < global_F) atomicAdd(&ps[ff[j]], dd[j] * cacc[j]);  // padding elements carry feature F
    }
}


// =========================================================== adjoint =====

// ------------------------------------------------- warp transpose-reduce --
//
// Each lane holds N values (N a power of two <= 32).  log2(N) halving steps
// exchange half of the values with the partner lane at distance 16, 8, ...,
// keeping the other half, so that after them lane L holds, summed over a group
// of lanes, the value with index L >> (5 - log2 N); the remaining distances
// finish the sum.  N - 1 + (5 - log2 N) shuffles instead of 5 N.
template <int N>
__device__ __forceinline__ float transpose_reduce(float (&v)[N], int lane) {
    static_assert(N >= 1 && N <= 32 && (N & (N - 1)) == 0, "N must be a power of two <= 32");
#pragma unroll
    for (int half = N / 2, off = 16; half >= 1; half >>= 1, off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    float r = v[0];
    constexpr int LOG = (N >= 32) ? 5 : (N >= 16) ? 4 : (N >= 8) ? 3 : (N >= 4) ? 2 : (N >= 2) ? 1 : 0;
#pragma unroll
    for (int off = (16 >> LOG); off >= 1; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    return r;
}

constexpr int pow2_at_least(int x) { return x <= 1 ? 1 : 2 * pow2_at_least((x + 1) / 2); }

// Reduce dz[0..D) and dval over the warp and add them to the FP64 accumulators.
// dval rides in the transpose-reduce when D + 1 fits the same power of two,
// otherwise it gets its own butterfly.
template <int D, typename T>
__device__ __forceinline__ void flush_path_grads(T (&dz)[D], T dval, int lane, double* g_slot_p,
                                                 double* g_val_p) {
    if constexpr (std::is_same<T, float>::value && D <= 32) {
        constexpr int NJ = pow2_at_least(D + 1);
        constexpr bool JOINT = NJ <= 32 && NJ == pow2_at_least(D);
        constexpr int N = JOINT ? NJ : pow2_at_least(D);
        constexpr int LOG = (N >= 32) ? 5 : (N >= 16) ? 4 : (N >= 8) ? 3 : (N >= 4) ? 2 : (N >= 2) ? 1 : 0;
        float v[N];
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = i < D ? dz[i] : ((JOINT && i == D) ? dval : 0.f);
        const float r = transpose_reduce<N>(v, lane);
        const int idx = lane >> (5 - LOG);
        if ((lane & ((1 << (5 - LOG)) - 1)) == 0) {
            if (idx < D) atomicAdd(&g_slot_p[idx], (double)r);
            else if (JOINT && idx == D) atomicAdd(g_val_p, (double)r);
        }
        if constexpr (!JOINT) {
            float x = dval;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0) atomicAdd(g_val_p, (double)x);
        }
    } else {
#pragma unroll
        for (int j = 0; j <= D; ++j) {
            T x = j < D ? dz[j] : dval;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0) {
                if (j < D) atomicAdd(&g_slot_p[j], (double)x);
                else atomicAdd(g_val_p, (double)x);
            }
        }
    }
}

// ------------------------------------------------------------------ FP32 --

// RECOMP: recompute a_j in the backward sweep instead of keeping it in
// registers (one more FMA per element and node, a third fewer registers).
template <int D, int NP, bool HAS_NAN, int PHI, bool RECOMP, typename XR, typename GR, bool PAIRS = false>
__device__ __forceinline__ void bwd_path_f32(const Rec32* __restrict__ r, const XR& xr, const GR& gr,
                                             float* ps, int lane, const QuadF& q, double* g_slot_p,
                                             double* g_val_p) {
    constexpr int K = NP / 2;
    constexpr int DA = RECOMP ? 1 : D;
    const float val = r[0].z;
    const bool pair = PAIRS && (r[D].bits & kPairElem) != 0;
    float dd[D], uu[D], acc1[D], acc2[D], acc3 = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Rec32 e = r[1 + j];
        const int f = feat_of(e.bits);
        const float x = xr(f);
        const bool o = satisfies<HAS_NAN>(x, e.lo, e.hi, e.bits);
        dd[j] = (o ? 1.f : 0.f) - e.z;
        if (j == D - 1 && pair) dd[j] = pair_d(x, e, r[0]);
        uu[j] = gr(f) * dd[j];
        acc1[j] = 0.f;
        acc2[j] = 0.f;
    }
    const int npass = q.n_pad / NP;
    for (int pass = 0; pass < npass; ++pass) {
        float2 T[K], C2[K], A[DA][K], P[D][K], PU[D][K], S[K], SU[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int m = pass * NP + 2 * k;
            T[k] = f2(q.t[m], q.t[m + 1]);
            C2[k] = f2(1.f - q.t[m], 1.f - q.t[m + 1]);
            P[0][k] = f2(q.w[m], q.w[m + 1]);
            PU[0][k] = f2s(0.f);
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float2 z2 = f2s(r[1 + j].z), d2 = f2s(dd[j]), u2 = f2s(uu[j]);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float2 a = fma2(T[k], d2, z2);
                if (!RECOMP) A[RECOMP ? 0 : j][k] = a;
                if (j + 1 < D) {
                    P[j + 1][k] = mul2(P[j][k], a);
                    PU[j + 1][k] = fma2(PU[j][k], a, mul2(u2, P[j][k]));
                }
            }
        }
        if constexpr (PAIRS && D > 1) {
#pragma unroll
            for (int k = 0; k < K; ++k) acc3 += PU[D - 1][k].x + PU[D - 1][k].y;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            S[k] = f2s(1.f);
            SU[k] = f2s(0.f);
        }
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            const float2 u2 = f2s(uu[j]);
            float2 a1 = mul2(P[j][0], S[0]);
            float2 a2 = mul2(C2[0], fma2(P[j][0], SU[0], mul2(PU[j][0], S[0])));
#pragma unroll
            for (int k = 1; k < K; ++k) {
                a1 = fma2(P[j][k], S[k], a1);
                a2 = fma2(C2[k], fma2(P[j][k], SU[k], mul2(PU[j][k], S[k])), a2);
            }
            if (j > 0) {
                float2 z2, d2;
                if (RECOMP) {
                    z2 = f2s(r[1 + j].z);
                    d2 = f2s(dd[j]);
                }
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float2 a = RECOMP ? fma2(T[k], d2, z2) : A[RECOMP ? 0 : j][k];
                    SU[k] = fma2(SU[k], a, mul2(u2, S[k]));
                    S[k] = mul2(S[k], a);
                }
            }
            acc1[j] += a1.x + a1.y;
            acc2[j] += a2.x + a2.y;
        }
    }
    float dval = 0.f, dz[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int f = feat_of(r[1 + j].bits);
        dval = fmaf(uu[j], acc1[j], dval);
        dz[j] = val * (acc2[j] - gr(f) * acc1[j]);
        phi_add<PHI>(ps, f * kTileLd + lane, val * dd[j] * acc1[j]);
    }
    if constexpr (PAIRS) {
        if (pair) {  // val = 1: dval becomes o_A K, a second sum o_B K goes to g_val_p[1]
            const Rec32 e = r[D];
            const int f = feat_of(e.bits);
            bool oa, ob;
            pair_sides(xr(f), e, r[0], &oa, &ob);
            const float k = acc3 - acc2[D - 1] + gr(f) * acc1[D - 1];
            dval = oa ? k : 0.f;
            float rb = ob ? k : 0.f;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) rb += __shfl_xor_sync(0xffffffffu, rb, off);
            if (lane == 0) atomicAdd(g_val_p + 1, (double)rb);
        }
    }
    flush_path_grads<D, float>(dz, dval, lane, g_slot_p, g_val_p);
}

// Packed variant: one node pair per pass, a_j recomputed, and everything the
// node loop touches kept as register pairs - {d_j, d_j}, {u_j, u_j} and the two
// per-element accumulators - so a pass issues only the 12 packed operations per
// element plus the z reload; the pair halves are added once after all passes.
template <int D, bool HAS_NAN, int PHI, typename XR, typename GR, bool PAIRS = false>
__device__ __forceinline__ void bwd_path_f32_pk(const Rec32* __restrict__ r, const XR& xr, const GR& gr,
                                                float* ps, int lane, const QuadF& q, double* g_slot_p,
                                                double* g_val_p) {
    const float val = r[0].z;
    const bool pair = PAIRS && (r[D].bits & kPairElem) != 0;
    float2 d2[D], u2[D], a1[D], a2[D], a3 = f2s(0.f);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Rec32 e = r[1 + j];
        const int f = feat_of(e.bits);
        const float x = xr(f);
        const bool o = satisfies<HAS_NAN>(x, e.lo, e.hi, e.bits);
        float d = (o ? 1.f : 0.f) - e.z;
        if (j == D - 1 && pair) d = pair_d(x, e, r[0]);
        d2[j] = f2s(d);
        u2[j] = f2s(gr(f) * d);
        a1[j] = f2s(0.f);
        a2[j] = f2s(0.f);
    }
    const int npass = q.n_pad / 2;
    for (int pass = 0; pass < npass; ++pass) {
        const int m = 2 * pass;
        const float2 T = f2(q.t[m], q.t[m + 1]);
        const float2 C2 = f2(1.f - q.t[m], 1.f - q.t[m + 1]);
        float2 P[D], PU[D];
        P[0] = f2(q.w[m], q.w[m + 1]);
        PU[0] = f2s(0.f);
#pragma unroll
        for (int j = 0; j + 1 < D; ++j) {
            const float2 a = fma2(T, d2[j], f2s(r[1 + j].z));
            P[j + 1] = mul2(P[j], a);
            PU[j + 1] = fma2(PU[j], a, mul2(u2[j], P[j]));
        }
        if constexpr (PAIRS && D > 1) a3 = add2(a3, PU[D - 1]);
        float2 S = f2s(1.f), SU = f2s(0.f);
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            a1[j] = fma2(P[j], S, a1[j]);
            a2[j] = fma2(C2, fma2(P[j], SU, mul2(PU[j], S)), a2[j]);
            if (j > 0) {
                const float2 a = fma2(T, d2[j], f2s(r[1 + j].z));
                SU = fma2(SU, a, mul2(u2[j], S));
                S = mul2(S, a);
            }
        }
    }
    float dval = 0.f, dz[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int f = feat_of(r[1 + j].bits);
        const float c1 = a1[j].x + a1[j].y, c2 = a2[j].x + a2[j].y;
        dval = fmaf(u2[j].x, c1, dval);
        dz[j] = val * (c2 - gr(f) * c1);
        phi_add<PHI>(ps, f * kTileLd + lane, val * d2[j].x * c1);
    }
    if constexpr (PAIRS) {
        if (pair) {  // val = 1: dval becomes o_A K, a second sum o_B K goes to g_val_p[1]
            const Rec32 e = r[D];
            const int f = feat_of(e.bits);
            bool oa, ob;
            pair_sides(xr(f), e, r[0], &oa, &ob);
            const float c1 = a1[D - 1].x + a1[D - 1].y, c2 = a2[D - 1].x + a2[D - 1].y;
            const float k = (a3.x + a3.y) - c2 + gr(f) * c1;
            dval = oa ? k : 0.f;
            float rb = ob ? k : 0.f;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) rb += __shfl_xor_sync(0xffffffffu, rb, off);
            if (lane == 0) atomicAdd(g_val_p + 1, (double)rb);
        }
    }
    flush_path_grads<D, float>(dz, dval, lane, g_slot_p, g_val_p);
}

// ------------------------------------------------- two samples per lane --
//
// Sample-pair packing: lane l handles samples 2l and 2l+1 of a 64-sample tile
// and every f32x2 operation covers the two samples at one quadrature node, so
// (o - z) and g (o - z) are natural pairs, the node sums need no horizontal
// adds, and the per-path setup and warp reduction serve 64 samples.
// {z_j, z_j} pairs come from this warp's shared scratch zs[0..D).
// The private phi tile has rows of kTileLd2 floats (lane l owns columns 2l, 2l+1).
constexpr int kTileLd2 = 66;

// 64-bit shared load that the compiler may not hoist out of the node loop
// (keeping all D pairs live would cost 2 D registers).
__device__ __forceinline__ float2 lds_pair(const float2* p) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(smem_u32(p)));
    return v;
}

struct GlobalCols2 {  // transposed global copy [feature][ld]; samples s, s+1 (s even)
    const float* t;
    int64_t ld;
    int64_t s;
    __device__ __forceinline__ float2 operator()(int f) const {
        return __ldg(reinterpret_cast<const float2*>(t + (int64_t)f * ld + s));
    }
};

template <int D, bool HAS_NAN, bool PAIRS = false>
__device__ __forceinline__ void bwd_path_f32_sp(const Rec32* __restrict__ r, const GlobalCols2& xr,
                                                const GlobalCols2& gr, float* ps, float2* zs, int lane,
                                                const QuadF& q, double* g_slot_p, double* g_val_p) {
    const float val = r[0].z;
    const bool pair = PAIRS && (r[D].bits & kPairElem) != 0;
    float2 d2[D], u2[D], a1[D], a2[D], a3 = f2s(0.f);
    __syncwarp();
    if (lane < D) zs[lane] = f2s(r[1 + lane].z);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Rec32 e = r[1 + j];
        const int f = feat_of(e.bits);
        const float2 x = xr(f);
        const bool oa = satisfies<HAS_NAN>(x.x, e.lo, e.hi, e.bits);
        const bool ob = satisfies<HAS_NAN>(x.y, e.lo, e.hi, e.bits);
        d2[j] = f2((oa ? 1.f : 0.f) - e.z, (ob ? 1.f : 0.f) - e.z);
        if (j == D - 1 && pair) d2[j] = f2(pair_d(x.x, e, r[0]), pair_d(x.y, e, r[0]));
        u2[j] = mul2(gr(f), d2[j]);
        a1[j] = f2s(0.f);
        a2[j] = f2s(0.f);
    }
    __syncwarp();
    for (int m = 0; m < q.n_pad; ++m) {
        const float2 T = f2s(q.t[m]);
        const float2 C2 = f2s(1.f - q.t[m]);
        float2 P[D], PU[D];
        P[0] = f2s(q.w[m]);
        PU[0] = f2s(0.f);
#pragma unroll
        for (int j = 0; j + 1 < D; ++j) {
            const float2 a = fma2(T, d2[j], lds_pair(zs + j));
            P[j + 1] = mul2(P[j], a);
            PU[j + 1] = fma2(PU[j], a, mul2(u2[j], P[j]));
        }
        if constexpr (PAIRS && D > 1) a3 = add2(a3, PU[D - 1]);
        float2 S = f2s(1.f), SU = f2s(0.f);
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            a1[j] = fma2(P[j], S, a1[j]);
            a2[j] = fma2(C2, fma2(P[j], SU, mul2(PU[j], S)), a2[j]);
            if (j > 0) {
                const float2 a = fma2(T, d2[j], lds_pair(zs + j));
                SU = fma2(SU, a, mul2(u2[j], S));
                S = mul2(S, a);
            }
        }
    }
    float2 dval2 = f2s(0.f);
    float dz[D];
    const float2 v2 = f2s(val);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int f = feat_of(r[1 + j].bits);
        dval2 = fma2(u2[j], a1[j], dval2);
        const float2 dzj = mul2(v2, fma2(f2s(-1.f), mul2(gr(f), a1[j]), a2[j]));
        dz[j] = dzj.x + dzj.y;
        float2* cell = reinterpret_cast<float2*>(ps + f * kTileLd2 + 2 * lane);
        *cell = fma2(mul2(v2, d2[j]), a1[j], *cell);  // private tile: plain read-add-write
    }
    if constexpr (PAIRS) {
        if (pair) {  // val = 1: dval becomes o_A K, a second sum o_B K goes to g_val_p[1]
            const Rec32 e = r[D];
            const int f = feat_of(e.bits);
            const float2 x = xr(f);
            bool oa0, ob0, oa1, ob1;
            pair_sides(x.x, e, r[0], &oa0, &ob0);
            pair_sides(x.y, e, r[0], &oa1, &ob1);
            const float2 k = fma2(gr(f), a1[D - 1], fma2(f2s(-1.f), a2[D - 1], a3));
            dval2 = f2(oa0 ? k.x : 0.f, oa1 ? k.y : 0.f);
            float rb = (ob0 ? k.x : 0.f) + (ob1 ? k.y : 0.f);
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) rb += __shfl_xor_sync(0xffffffffu, rb, off);
            if (lane == 0) atomicAdd(g_val_p + 1, (double)rb);
        }
    }
    flush_path_grads<D, float>(dz, dval2.x + dval2.y, lane, g_slot_p, g_val_p);
}

// ------------------------------------------------------------------ FP64 --

template <int D, bool HAS_NAN>
__device__ __forceinline__ void bwd_path_f64(const Rec64* __restrict__ r, const float* __restrict__ xs,
                                             const float* __restrict__ gs, int lane, const QuadD& q,
                                             double* g_slot_p, double* g_val_p) {
    const double val = r[0].z;
    double dd[D], uu[D], acc1[D], acc2[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Rec64 e = r[1 + j];
        const int f = feat_of(e.bits);
        const float x = xs[f * kTileLd + lane];
        const bool o = satisfies<HAS_NAN>(x, e.lo, e.hi, e.bits);
        dd[j] = (o ? 1.0 : 0.0) - e.z;
        uu[j] = (double)gs[f * kTileLd + lane] * dd[j];
        acc1[j] = acc2[j] = 0.0;
    }
    for (int m = 0; m < q.n; ++m) {
        const double t = q.t[m];
        double A[D], P[D], PU[D];
        P[0] = q.w[m];
        PU[0] = 0.0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            A[j] = fma(t, dd[j], r[1 + j].z);
            if (j + 1 < D) {
                P[j + 1] = P[j] * A[j];
                PU[j + 1] = fma(PU[j], A[j], uu[j] * P[j]);
            }
        }
        double S = 1.0, SU = 0.0;
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            acc1[j] = fma(P[j], S, acc1[j]);
            acc2[j] = fma(1.0 - t, fma(P[j], SU, PU[j] * S), acc2[j]);
            SU = fma(SU, A[j], uu[j] * S);
            S *= A[j];
        }
    }
    double dval = 0.0, dz[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int f = feat_of(r[1 + j].bits);
        dval = fma(uu[j], acc1[j], dval);
        dz[j] = val * (acc2[j] - (double)gs[f * kTileLd + lane] * acc1[j]);
    }
    flush_path_grads<D, double>(dz, dval, lane, g_slot_p, g_val_p);
}


}  // namespace qts
