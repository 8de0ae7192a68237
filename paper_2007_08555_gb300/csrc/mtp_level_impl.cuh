// Kernels of one lev_max, instantiated by a generated translation unit that first includes the
// generated header and defines MTP_GEN_NS (its namespace) and MTP_LEVEL_FN (registry function).
//
// One evaluation (Sec. 2.1, Eqs. 1-4) runs four kernels:
//   k_moments   thread group per atom: radial functions f_mu (Eq. 3 with the Chebyshev basis of
//               Eq. 4) and the symmetric moment components M_{mu,nu}[a,b,c] = sum_j f_mu x^a y^b z^c,
//               accumulated in registers slice by slice (the slices are generated, unrolled code);
//   k_contract  warp per atom: the generated contraction program (every basis function B_alpha),
//               the site energy V_i = sum xi_alpha B_alpha (Eq. 2), then the adjoint program
//               dV_i/dM, all in shared memory (FP64 path); the float path runs the program in
//               parts instead (k_contract_parts: one warp per part and 32 atoms);
//   k_pairgrad  thread group per atom: dV_i/dr_ij = sum adj * d(f_mu(r) mono(r))/dr per pair, with
//               dV_i/dM staged in shared memory on the float path;
//   k_gather    thread group per atom: F_i = sum_p (g_ip - g_{j_p, reverse}) and the virial
//               W = -sum g_ij (x) r_ij, summed per warp and added per configuration in double.
// The kernels of one evaluation are chained by programmatic dependent launch (launch_pdl).
#include "mtp_common.cuh"
#include "mtp_level.h"

namespace mtp {
namespace MTP_GEN_NS {

using G = ::MTP_GEN_NS::Traits;

template <class T, int S>
struct SliceSel;
template <int S>
struct SliceSel<float, S> {
    using type = typename G::template F32<S>;
};
template <int S>
struct SliceSel<double, S> {
    using type = typename G::template F64<S>;
};
template <class T>
struct NumSlices;
template <>
struct NumSlices<float> {
    static constexpr int value = G::NS32_;
};
template <>
struct NumSlices<double> {
    static constexpr int value = G::NS64_;
};
// slices of the moments kernel: in float as many as above with balanced sizes (the largest slice
// sets the running sums a thread holds), in double the same as above
template <class T, int S>
struct MomSliceSel;
template <int S>
struct MomSliceSel<float, S> {
    using type = typename G::template MF32<S>;
};
template <int S>
struct MomSliceSel<double, S> {
    using type = typename G::template F64<S>;
};
template <class T>
struct NumMomSlices;
template <>
struct NumMomSlices<float> {
    static constexpr int value = G::NSM32_;
};
template <>
struct NumMomSlices<double> {
    static constexpr int value = G::NS64_;
};

__device__ __forceinline__ int clamp_species(int z, int S) { return z < 0 ? 0 : (z >= S ? S - 1 : z); }
__device__ __forceinline__ float my_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double my_sqrt(double x) { return sqrt(x); }

// Double-float numbers (hi + lo, |lo| <= ulp(hi) / 2): Knuth's TwoSum and the FMA form of Dekker's
// TwoProduct give the exact rounding errors, so sums and products keep ~44 significant bits on the
// FP32 pipe (GB300 issues double precision at a small fraction of the FP32 rate).
struct Df {
    float hi, lo;
};
__device__ __forceinline__ Df df_norm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ Df df_add(Df a, Df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return df_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ Df df_mul(Df a, Df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    return df_norm(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}
__device__ __forceinline__ Df df_mulf(Df a, float b) {
    const float p = __fmul_rn(a.hi, b);
    const float e = __fmaf_rn(a.hi, b, -p);
    return df_norm(p, __fmaf_rn(a.lo, b, e));
}
__device__ __forceinline__ Df df_neg(Df a) { return {-a.hi, -a.lo}; }

// Radial coefficients in shared memory: per ordered species pair a block [b][mu] with mu padded to
// a whole vector (4 floats or 2 doubles), so that the N_mu coefficients of one Chebyshev order come
// in one or two vector loads.
template <class T>
struct CoefPad {
    static constexpr int value = sizeof(T) == 4 ? ((G::NMU_ + 3) & ~3) : ((G::NMU_ + 1) & ~1);
};

template <class T>
__device__ __forceinline__ void coefs_at(const T* __restrict__ cz, int b, T* out) {
    constexpr int P = CoefPad<T>::value;
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < P / 4; ++k) {
            const float4 v = reinterpret_cast<const float4*>(cz + b * P)[k];
            out[4 * k] = v.x;
            out[4 * k + 1] = v.y;
            out[4 * k + 2] = v.z;
            out[4 * k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < P / 2; ++k) {
            const double2 v = reinterpret_cast<const double2*>(cz + b * P)[k];
            out[2 * k] = v.x;
            out[2 * k + 1] = v.y;
        }
    }
}

// The radial functions (Eq. 3) and their derivatives in double-float arithmetic, rounded to float at
// the end: below R_min the Chebyshev polynomials leave [-1, 1] and grow, and their float sum loses
// the digits that this evaluation keeps.
template <bool WANT_D>
__device__ __forceinline__ void radial_df(const float r, const float* __restrict__ cz, const int NQ, const float rmin,
                                       const float rcut, float* f, float* df) {
    constexpr int NMU = G::NMU_;
    // x = (2 r - R_min - R_cut) / (R_cut - R_min)
    const Df span = df_add({rcut, 0.f}, {-rmin, 0.f});
    const Df num = df_add(df_add({2.f * r, 0.f}, {-rmin, 0.f}), {-rcut, 0.f});
    const float q = num.hi / span.hi;
    const Df rem = df_add(num, df_neg(df_mulf(span, q)));  // num - q span
    const Df x = df_add({q, 0.f}, {rem.hi / span.hi, 0.f});
    const Df x2 = {2.f * x.hi, 2.f * x.lo};
    Df F[NMU], D[NMU];
    float cb[CoefPad<float>::value];
    coefs_at(cz, 0, cb);
#pragma unroll
    for (int mu = 0; mu < NMU; ++mu) {
        F[mu] = {cb[mu], 0.f};
        D[mu] = {0.f, 0.f};
    }
    Df t0 = {1.f, 0.f}, t1 = x, d0 = {0.f, 0.f}, d1 = {1.f, 0.f};
    for (int b = 1; b < NQ; ++b) {
        Df tb = t1, db = d1;
        if (b > 1) {  // T_b = 2 x T_{b-1} - T_{b-2};  T_b' = 2 T_{b-1} + 2 x T_{b-1}' - T_{b-2}'
            tb = df_add(df_mul(x2, t1), df_neg(t0));
            if (WANT_D) db = df_add(df_add({2.f * t1.hi, 2.f * t1.lo}, df_mul(x2, d1)), df_neg(d0));
            t0 = t1;
            t1 = tb;
            if (WANT_D) {
                d0 = d1;
                d1 = db;
            }
        }
        coefs_at(cz, b, cb);
#pragma unroll
        for (int mu = 0; mu < NMU; ++mu) {
            F[mu] = df_add(F[mu], df_mulf(tb, cb[mu]));
            if (WANT_D) D[mu] = df_add(D[mu], df_mulf(db, cb[mu]));
        }
    }
    // Q = T (R_cut - r)^2;  dQ/dr = T' (2 / span) (R_cut - r)^2 - 2 T (R_cut - r)
    const Df u = df_add({rcut, 0.f}, {-r, 0.f});
    const Df u2 = df_mul(u, u);
    const float two_over_span = 2.f / span.hi;
#pragma unroll
    for (int mu = 0; mu < NMU; ++mu) {
        const Df fu = df_mul(F[mu], u2);
        f[mu] = fu.hi + fu.lo;
        if (WANT_D) {
            const Df d = df_add(df_mulf(df_mul(D[mu], u2), two_over_span), df_mulf(df_mul(F[mu], u), -2.f));
            df[mu] = d.hi + d.lo;
        }
    }
}

// f_mu(r) = (R_cut - r)^2 sum_b c_b T_b(x) and its r-derivative (Eqs. 3-4); Chebyshev T_b by the
// three-term recurrence, dT_b/dx by its derivative.  cz points at c[z_i][z_j][0][0].
// Below R_min the Chebyshev polynomials leave [-1, 1], grow quickly and cancel in the sum; there the
// float evaluation alone costs the float path ~1e-5 in the energy, so the float path takes those
// (rare) pairs through radial_df; the common case stays plain float.
template <class T, bool WANT_D>
__device__ __forceinline__ void radial(const T r, const T* __restrict__ cz, const int NQ, const T rmin,
                                       const T rcut, const T inv_span, T* f, T* df) {
    constexpr int NMU = G::NMU_;
    if constexpr (sizeof(T) == 4) {
        if (r < rmin) {
            radial_df<WANT_D>(r, cz, NQ, rmin, rcut, f, df);
            return;
        }
    }
    const T x = (T(2) * r - rmin - rcut) * inv_span;
    T F[NMU], D[NMU];
    T cb[CoefPad<T>::value];
    coefs_at(cz, 0, cb);
#pragma unroll
    for (int mu = 0; mu < NMU; ++mu) {
        F[mu] = cb[mu];
        D[mu] = T(0);
    }
    if (NQ > 1) {
        coefs_at(cz, 1, cb);
#pragma unroll
        for (int mu = 0; mu < NMU; ++mu) {
            F[mu] += cb[mu] * x;
            if (WANT_D) D[mu] += cb[mu];
        }
    }
    T t0 = T(1), t1 = x, d0 = T(0), d1 = T(1);
    for (int b = 2; b < NQ; ++b) {
        const T t2 = T(2) * x * t1 - t0;
        const T d2 = T(2) * t1 + T(2) * x * d1 - d0;
        coefs_at(cz, b, cb);
#pragma unroll
        for (int mu = 0; mu < NMU; ++mu) {
            F[mu] += cb[mu] * t2;
            if (WANT_D) D[mu] += cb[mu] * d2;
        }
        t0 = t1;
        t1 = t2;
        d0 = d1;
        d1 = d2;
    }
    // Q_b = 0 for r >= R_cut (Eq. 4): pairs kept in a neighbour list with a skin contribute nothing
    const T u = r < rcut ? rcut - r : T(0);
    const T u2 = u * u;
#pragma unroll
    for (int mu = 0; mu < NMU; ++mu) {
        f[mu] = F[mu] * u2;
        if (WANT_D) df[mu] = D[mu] * (T(2) * inv_span) * u2 - T(2) * F[mu] * u;
    }
}

// Elements between the coefficient rows of two species pairs: one 16-byte vector more than the row,
// so that lanes reading the same Chebyshev order for different species pairs hit different banks.
template <class T>
__host__ __device__ inline int coef_row(const EvalCtx<T>& a) {
    return CoefPad<T>::value * a.NQ + 16 / (int)sizeof(T);
}

template <class T>
__device__ __forceinline__ void load_c(const EvalCtx<T>& a, T* cs) {
    // global c[z_i][z_j][mu][b] -> shared [z_i][z_j][b][mu padded], rows coef_row apart
    constexpr int P = CoefPad<T>::value;
    const int row = coef_row(a);
    const int nc = a.S * a.S * row;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
        const int pair = k / row, e = k % row;
        const int mu = e % P, b = e / P;
        cs[k] = (mu < G::NMU_ && b < a.NQ) ? a.c[((size_t)pair * G::NMU_ + mu) * a.NQ + b] : T(0);
    }
    __syncthreads();
}

// bytes of the shared coefficient table
template <class T>
__host__ __device__ inline size_t coef_bytes(const EvalCtx<T>& a) {
    return sizeof(T) * (size_t)a.S * a.S * coef_row(a);
}

// ----------------------------------------------------------------------------------------------
// k_moments
// ----------------------------------------------------------------------------------------------
// one pair's inputs: r_ij and the neighbour's species
template <class T>
struct PairIn {
    T x, y, z;
    int zj;
};
template <class T>
__device__ __forceinline__ PairIn<T> load_pair(const EvalCtx<T>& a, size_t idx) {
    const PairRec<T> q = a.pr[idx];
    return PairIn<T>{q.x, q.y, q.z, q.jz >> 24};
}

template <class T, int S, int TPA>
__device__ __forceinline__ void moments_slice(const EvalCtx<T>& a, int i, int sub, bool active, int zi, int cnt,
                                              const T* cs) {
    using SL = typename MomSliceSel<T, S>::type;
    T acc[SL::SIZE];
#pragma unroll
    for (int t = 0; t < SL::SIZE; ++t) acc[t] = T(0);
    const size_t n = (size_t)a.n_atoms;
    if (active) {
        const int csz = coef_row(a);
        // the pair records two steps ahead are in flight during this pair's arithmetic (one record
        // is one wide load that spans several cache lines of the slot-major rows)
        PairIn<T> nx1 = load_pair(a, sub < cnt ? (size_t)sub * n + i : (size_t)i);
        PairIn<T> nx2 = load_pair(a, sub + TPA < cnt ? (size_t)(sub + TPA) * n + i : (size_t)i);
        for (int p = sub; p < cnt; p += TPA) {
            const PairIn<T> cur = nx1;
            nx1 = nx2;
            if (p + 2 * TPA < cnt) nx2 = load_pair(a, (size_t)(p + 2 * TPA) * n + i);
            const T x = cur.x, y = cur.y, z = cur.z;
            const T r = my_sqrt(x * x + y * y + z * z);
            T f[G::NMU_];
            radial<T, false>(r, cs + (zi * a.S + cur.zj) * csz, a.NQ, a.rmin, a.rcut, a.inv_span, f, nullptr);
            SL::template mom<T>(x, y, z, f, acc);
        }
    }
    if (TPA > 1) {
#pragma unroll
        for (int t = 0; t < SL::SIZE; ++t) {
#pragma unroll
            for (int o = 1; o < TPA; o <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
        }
    }
    if (active) {
        // the group's lanes store disjoint parts of the slice (tile layout [tile][C][32])
        T* dst = a.mom + (size_t)(i >> 5) * G::C_ * 32 + (i & 31);
#pragma unroll
        for (int t = 0; t < SL::SIZE; ++t)
            if (t % TPA == sub) dst[(size_t)(SL::BEGIN + t) * 32] = acc[t];
    }
}

template <class T, int S, int NS, int TPA>
__device__ __forceinline__ void moments_all(const EvalCtx<T>& a, int i, int sub, bool active, int zi, int cnt,
                                            const T* cs) {
    if constexpr (S < NS) {
        moments_slice<T, S, TPA>(a, i, sub, active, zi, cnt, cs);
        moments_all<T, S + 1, NS, TPA>(a, i, sub, active, zi, cnt, cs);
    }
}

template <class T, int TPA>
__global__ void __launch_bounds__(128) k_moments(const EvalCtx<T> a) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* cs = reinterpret_cast<T*>(smem_raw);
    load_c(a, cs);
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    // the first evaluation kernel clears the per-configuration sums (energy, virial) that later
    // kernels accumulate
    for (int t = gtid; t < 10 * a.n_cfg; t += stride) {
        if (t < a.n_cfg) {
            if (a.energy) a.energy[t] = 0.0;
        } else if (a.virial) {
            a.virial[t - a.n_cfg] = 0.0;
        }
    }
    // packed-atom work queue: every warp takes the next 32 (atom, lane) units of the batch (atoms of
    // all configurations in one sequence) until none are left; whole warps stay converged
    const int total = ((a.n_atoms + 31) / 32) * 32 * TPA;
    const int lane = threadIdx.x & 31;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(a.queue, 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total) break;
        const int g = base + lane;
        const int i = g / TPA, sub = g % TPA;
        const bool active = i < a.n_atoms;
        int zi = 0, cnt = 0;
        if (active) {
            zi = clamp_species(a.types[i], a.S);  // out-of-range species are reported by the neighbour build
            cnt = a.count[i];
        }
        moments_all<T, 0, NumMomSlices<T>::value, TPA>(a, i, sub, active, zi, cnt, cs);
    }
}

// ----------------------------------------------------------------------------------------------
// k_contract: warp per atom
// ----------------------------------------------------------------------------------------------
// One layer-ordered pass of a generated program over A atoms held by the warp.  Op word layout:
// i (16) | j (16) | k (16) | flags (3) | weight index (13); flags: 1 = first term of the target,
// 2 = last term (store), 4 = padding.  Forward: val[k] = sum w val[i] val[j].  Adjoint:
// adj[k] = adj[k] + sum w val[i] adj[j] (the target's own seed enters through the first term).
template <class T, int A, bool ADJ>
__device__ __forceinline__ void run_program(const unsigned long long* __restrict__ ops, const int* __restrict__ layer_end,
                                            int layers, const float* sw, T* val, T* adj, int lane) {
    constexpr int V = G::V_;
    int row = 0;
    for (int l = 0; l < layers; ++l) {
        const int end = layer_end[l];
        T acc[A];
#pragma unroll
        for (int q = 0; q < A; ++q) acc[q] = T(0);
        unsigned long long op = row < end ? ops[row * 32 + lane] : 4ull << 48;
        for (; row < end; ++row) {
            const unsigned long long nxt = row + 1 < end ? ops[(row + 1) * 32 + lane] : 4ull << 48;  // prefetch
            const unsigned fl = (unsigned)(op >> 48) & 7u;
            if (!(fl & 4u)) {
                const int i = (int)(op & 0xffffu), j = (int)((op >> 16) & 0xffffu), k = (int)((op >> 32) & 0xffffu);
                const T w = (T)sw[op >> 51];
#pragma unroll
                for (int q = 0; q < A; ++q) {
                    if (fl & 1u) acc[q] = ADJ ? adj[q * V + k] : T(0);
                    acc[q] += w * val[q * V + i] * (ADJ ? adj[q * V + j] : val[q * V + j]);
                    if (fl & 2u) {
                        if (ADJ)
                            adj[q * V + k] = acc[q];
                        else
                            val[q * V + k] = acc[q];
                    }
                }
            }
            op = nxt;
        }
        __syncwarp();
    }
}

// Flush a running per-configuration sum.
__device__ __forceinline__ void flush_sum(double* dst, int cfg, double v) {
    if (cfg >= 0 && dst) atomicAdd(&dst[cfg], v);
}

// warp per group of A consecutive atoms (contiguous chunks per warp)
template <class T, int A>
__global__ void __launch_bounds__(256) k_contract(const EvalCtx<T> a) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int V = G::V_, C = G::C_, M = G::M_;
    constexpr int MB = (M + 31) / 32;  // basis values per lane
    __shared__ int s_cfg[8];
    __shared__ double s_sum[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    T* seed = reinterpret_cast<T*>(smem_raw);
    float* sw = reinterpret_cast<float*>(seed + V);
    T* val = reinterpret_cast<T*>(sw + ((a.n_weights + 3) & ~3)) + (size_t)warp * 2 * A * V;
    T* adj = val + A * V;
    for (int v = threadIdx.x; v < V; v += blockDim.x) seed[v] = a.seed[v];
    for (int v = threadIdx.x; v < a.n_weights; v += blockDim.x) sw[v] = a.weights[v];
    __syncthreads();
    const int total_warps = gridDim.x * wpb;
    const int chunk = (a.n_atoms + total_warps - 1) / total_warps;
    const int gw = blockIdx.x * wpb + warp;
    const int i0 = gw * chunk;
    const int i1 = min(a.n_atoms, i0 + chunk);
    double esum = 0.0;
    int ecfg = -1;
    double brun[MB];
#pragma unroll
    for (int t = 0; t < MB; ++t) brun[t] = 0.0;
    for (int ib = i0; ib < i1; ib += A) {
        const int na = min(A, i1 - ib);
#pragma unroll
        for (int q = 0; q < A; ++q) {
            if (q < na) {
                const int i = ib + q;
                const T* msrc = a.mom + (size_t)(i >> 5) * C * 32 + (i & 31);
                for (int c = lane; c < C; c += 32) val[q * V + c] = msrc[(size_t)c * 32];
            }
        }
        __syncwarp();
        run_program<T, A, false>(a.fwd_ops, a.fwd_layer_end, a.fwd_layers, sw, val, adj, lane);
        for (int q = 0; q < na; ++q) {
            const int i = ib + q;
            const int cfg = a.cfg_of[i];
            if (cfg != ecfg) {  // warp-uniform
                if (lane == 0) flush_sum(a.energy, ecfg, esum);
                if (a.b_rows && ecfg >= 0) {
#pragma unroll
                    for (int t = 0; t < MB; ++t)
                        if (lane + 32 * t < M) atomicAdd(&a.b_rows[(size_t)ecfg * M + lane + 32 * t], brun[t]);
                }
#pragma unroll
                for (int t = 0; t < MB; ++t) brun[t] = 0.0;
                ecfg = cfg;
                esum = 0.0;
            }
            T e = T(0);
#pragma unroll
            for (int t = 0; t < MB; ++t) {
                const int al = lane + 32 * t;
                if (al < M) {
                    const T b = val[q * V + a.basis_value[al]];
                    e += a.xi[al] * b;
                    if (a.b_rows) brun[t] += (double)b;
                    if (a.b_atoms) a.b_atoms[(size_t)i * M + al] = (double)b;
                }
            }
            const double ed = warp_sum((double)e);
            if (lane == 0 && a.site) a.site[i] = ed;
            esum += ed;
        }
        for (int v = lane; v < A * V; v += 32) adj[v] = seed[v % V];
        __syncwarp();
        run_program<T, A, true>(a.adj_ops, a.adj_layer_end, a.adj_layers, sw, val, adj, lane);
#pragma unroll
        for (int q = 0; q < A; ++q) {
            if (q < na) {
                const int i = ib + q;
                T* adst = a.adjm + (size_t)(i >> 5) * C * 32 + (i & 31);
                for (int c = lane; c < C; c += 32) adst[(size_t)c * 32] = adj[q * V + c];
            }
        }
        __syncwarp();
    }
    if (a.b_rows && ecfg >= 0) {
#pragma unroll
        for (int t = 0; t < MB; ++t)
            if (lane + 32 * t < M) atomicAdd(&a.b_rows[(size_t)ecfg * M + lane + 32 * t], brun[t]);
    }
    // combine the warps' last running energies: one atomic per configuration per block
    if (lane == 0) {
        s_cfg[warp] = ecfg;
        s_sum[warp] = esum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int cur = -1;
        double acc = 0.0;
        for (int w = 0; w < wpb; ++w) {
            if (s_cfg[w] < 0) continue;
            if (s_cfg[w] != cur) {
                flush_sum(a.energy, cur, acc);
                cur = s_cfg[w];
                acc = 0.0;
            }
            acc += s_sum[w];
        }
        flush_sum(a.energy, cur, acc);
    }
}

#if MTPGEN_HAS_PARTS
// Float contraction, split into NPART generated parts (basis functions grouped so that one part's
// values fit in registers): warp w runs part w / n_tiles for the 32 atoms of tile w % n_tiles, so
// that the warps on an SM mostly run the same code.  Each part writes its site-energy share and
// dV/dM of its moments to slots; the pair-gradient kernel adds the slots of each component and the
// gather the energy shares, in a fixed order.
__global__ void __launch_bounds__(128) k_contract_parts(const EvalCtx<float> a) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int n_tiles = (a.n_atoms + 31) >> 5;
    const int total = n_tiles * G::NPART_;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += (gridDim.x * blockDim.x) >> 5) {
        const int part = w / n_tiles, tile = w - part * n_tiles;
        const int i = tile * 32 + lane;
        if (i >= a.n_atoms) continue;
        const float* src = a.mom + (size_t)tile * G::C_ * 32 + lane;
        float* dst = a.aslots + (size_t)tile * G::NSLOT_ * 32 + lane;
        double* bout = a.b_atoms ? a.b_atoms + (size_t)i * G::M_ : nullptr;
        const float e = bout ? ::MTP_GEN_NS::contract_part<true>(part, src, dst, a.xi, bout)
                             : ::MTP_GEN_NS::contract_part<false>(part, src, dst, a.xi, nullptr);
        a.epart[(size_t)part * a.n_atoms + i] = e;
    }
}

#endif

// b rows as sums of the per-atom rows of each configuration (one block per configuration)
template <class T>
__global__ void k_brows(const EvalCtx<T> a, const int* cfg_off) {
    pdl_enter();
    constexpr int M = G::M_;
    const int k = blockIdx.x;
    const int i0 = cfg_off[k], i1 = cfg_off[k + 1];
    for (int al = threadIdx.x; al < M; al += blockDim.x) {
        double s = 0.0;
        for (int i = i0; i < i1; ++i) s += a.b_atoms[(size_t)i * M + al];
        a.b_rows[(size_t)k * M + al] = s;
    }
}

// ----------------------------------------------------------------------------------------------
// k_pairgrad: g_ij = dV_i/dr_ij
// ----------------------------------------------------------------------------------------------
// dV/dM of one atom held in shared memory: components 4k .. 4k+3 in the vector q[k * NS] (NS atoms
// per block); repeated reads of one vector are merged by the compiler (no stores in between)
template <class T, int NS, int OFF = 0>
struct SharedAdj {
    const Vec4<T>* q;
    __device__ __forceinline__ T operator[](int t) const {
        const Vec4<T> v = q[((t + OFF) >> 2) * NS];
        const int c = (t + OFF) & 3;
        return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
    }
};

// the float path keeps dV/dM in shared memory, shared by the TPA lanes of an atom, which leaves
// the registers to the per-pair arithmetic (more resident warps); the double path keeps them in
// registers
template <class T>
struct PairgradShared {
#if MTPGEN_HAS_PARTS
    static constexpr bool value = sizeof(T) == 4;
#else
    static constexpr bool value = false;
#endif
};

// With two or more lanes per atom (PairgradMerged) dV/dM of every slice of an atom sits in shared
// memory at once and each pair is visited once: its record, radial functions and gradient store are
// not repeated per slice.  With one lane per atom a block holds 128 atoms and that array would not
// fit beside the coefficients at the largest sizes, so the slices take turns.
template <class T, int TPA>
struct PairgradMerged {
    static constexpr bool value = PairgradShared<T>::value && TPA >= 2 && NumSlices<T>::value > 1;
};

template <class T, int TPA>
constexpr size_t pairgrad_adj_bytes() {
    return !PairgradShared<T>::value ? 0
           : sizeof(T) * (size_t)(((PairgradMerged<T, TPA>::value ? G::C_ : G::MAXS32_) + 3) / 4 * 4) * (128 / TPA);
}

template <class T, int S, int TPA, class A>
__device__ __forceinline__ void pairgrad_pairs(const EvalCtx<T>& a, int i, int sub, int zi, int cnt, const T* cs,
                                               const A adj) {
    const size_t n = (size_t)a.n_atoms;
    const int csz = coef_row(a);
    // the next pair's loads are issued before this pair's arithmetic (their latency overlaps it)
    PairIn<T> nx{};
    if (sub < cnt) nx = load_pair(a, (size_t)sub * n + i);
#pragma unroll 1
    for (int p = sub; p < cnt; p += TPA) {
        const size_t idx = (size_t)p * n + i;
        const PairIn<T> cur = nx;
        if (p + TPA < cnt) nx = load_pair(a, (size_t)(p + TPA) * n + i);
        const T x = cur.x, y = cur.y, z = cur.z;
        const T r = my_sqrt(x * x + y * y + z * z);
        T f[G::NMU_], df[G::NMU_];
        radial<T, true>(r, cs + (zi * a.S + cur.zj) * csz, a.NQ, a.rmin, a.rcut, a.inv_span, f, df);
        T s = T(0), gx = T(0), gy = T(0), gz = T(0);
        SliceSel<T, S>::type::template grad<T>(x, y, z, f, df, adj, s, gx, gy, gz);
        const T sr = s / r;
        gx += sr * x;
        gy += sr * y;
        gz += sr * z;
        if (S == 0) {
            a.g[idx] = Vec4<T>{gx, gy, gz, T(0)};
        } else {
            const Vec4<T> o = a.g[idx];
            a.g[idx] = Vec4<T>{o.x + gx, o.y + gy, o.z + gz, T(0)};
        }
    }
}

template <class T, int S, int TPA>
__device__ __forceinline__ void pairgrad_slice(const EvalCtx<T>& a, int i, int sub, bool active, int zi, int cnt,
                                               const T* cs, T* sadj) {
    using SL = typename SliceSel<T, S>::type;
#if MTPGEN_HAS_PARTS
    if constexpr (PairgradShared<T>::value) {
        // dV/dM straight from the contraction parts' slots, summed in slot order, written once per
        // atom (its lanes share the work) and read by all of them
        constexpr int NSA = 128 / TPA;
        T* mine = sadj + 4 * (threadIdx.x / TPA);
        __syncwarp();  // the atom's lanes are done with the previous slice or atom
        if (active) SL::template adj_to_shared<T, TPA, NSA>(a.aslots + (size_t)(i >> 5) * G::NSLOT_ * 32 + (i & 31),
                                                            mine, sub);
        __syncwarp();
        pairgrad_pairs<T, S, TPA>(a, i, sub, zi, cnt, cs,
                                  SharedAdj<T, NSA>{reinterpret_cast<const Vec4<T>*>(mine)});
        return;
    }
#endif
    // (an inactive lane's atom index stays within the last tile, which is allocated in full)
    T adjs[SL::SIZE];
    const T* src = a.adjm + (size_t)(i >> 5) * G::C_ * 32 + (i & 31);
#pragma unroll
    for (int t = 0; t < SL::SIZE; ++t) adjs[t] = src[(size_t)(SL::BEGIN + t) * 32];
    pairgrad_pairs<T, S, TPA>(a, i, sub, zi, cnt, cs, adjs);
}

#if MTPGEN_HAS_PARTS
// dV/dM of every slice of the atom into its shared array, at the components' positions
template <class T, int S, int TPA, int NSA>
__device__ __forceinline__ void adj_all_to_shared(const T* sl, T* mine, int sub) {
    if constexpr (S < NumSlices<T>::value) {
        using SL = typename SliceSel<T, S>::type;
        SL::template adj_to_shared<T, TPA, NSA, SL::BEGIN>(sl, mine, sub);
        adj_all_to_shared<T, S + 1, TPA, NSA>(sl, mine, sub);
    }
}

// the adjoint terms of every slice for one pair
template <class T, int S, int NSA>
__device__ __forceinline__ void grad_all_slices(const T x, const T y, const T z, const T* f, const T* df,
                                                const Vec4<T>* q, T& s, T& gx, T& gy, T& gz) {
    if constexpr (S < NumSlices<T>::value) {
        using SL = typename SliceSel<T, S>::type;
        SL::template grad<T>(x, y, z, f, df, SharedAdj<T, NSA, SL::BEGIN>{q}, s, gx, gy, gz);
        grad_all_slices<T, S + 1, NSA>(x, y, z, f, df, q, s, gx, gy, gz);
    }
}

// every pair of the atom once, with all slices' adjoint terms (PairgradMerged)
template <class T, int TPA>
__device__ __forceinline__ void pairgrad_merged(const EvalCtx<T>& a, int i, int sub, bool active, int zi, int cnt,
                                                const T* cs, T* sadj) {
    constexpr int NSA = 128 / TPA;
    T* mine = sadj + 4 * (threadIdx.x / TPA);
    __syncwarp();  // the atom's lanes are done with the previous atom
    if (active)
        adj_all_to_shared<T, 0, TPA, NSA>(a.aslots + (size_t)(i >> 5) * G::NSLOT_ * 32 + (i & 31), mine, sub);
    __syncwarp();
    const Vec4<T>* q = reinterpret_cast<const Vec4<T>*>(mine);
    const size_t n = (size_t)a.n_atoms;
    const int csz = coef_row(a);
    PairIn<T> nx{};
    if (sub < cnt) nx = load_pair(a, (size_t)sub * n + i);
#pragma unroll 1
    for (int p = sub; p < cnt; p += TPA) {
        const size_t idx = (size_t)p * n + i;
        const PairIn<T> cur = nx;
        if (p + TPA < cnt) nx = load_pair(a, (size_t)(p + TPA) * n + i);
        const T x = cur.x, y = cur.y, z = cur.z;
        const T r = my_sqrt(x * x + y * y + z * z);
        T f[G::NMU_], df[G::NMU_];
        radial<T, true>(r, cs + (zi * a.S + cur.zj) * csz, a.NQ, a.rmin, a.rcut, a.inv_span, f, df);
        T s = T(0), gx = T(0), gy = T(0), gz = T(0);
        grad_all_slices<T, 0, NSA>(x, y, z, f, df, q, s, gx, gy, gz);
        const T sr = s / r;
        a.g[idx] = Vec4<T>{gx + sr * x, gy + sr * y, gz + sr * z, T(0)};
    }
}
#endif

template <class T, int S, int NS, int TPA>
__device__ __forceinline__ void pairgrad_all(const EvalCtx<T>& a, int i, int sub, bool active, int zi, int cnt,
                                             const T* cs, T* sadj) {
    if constexpr (S < NS) {
        pairgrad_slice<T, S, TPA>(a, i, sub, active, zi, cnt, cs, sadj);
        pairgrad_all<T, S + 1, NS, TPA>(a, i, sub, active, zi, cnt, cs, sadj);
    }
}

template <class T, int TPA>
__global__ void __launch_bounds__(128) k_pairgrad(const EvalCtx<T> a) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* cs = reinterpret_cast<T*>(smem_raw);
    T* sadj = reinterpret_cast<T*>(smem_raw + ((coef_bytes(a) + 15) & ~(size_t)15));
    load_c(a, cs);
    // the work queue of k_moments (a second counter): whole warps stay converged for __syncwarp
    const int total = ((a.n_atoms + 31) / 32) * 32 * TPA;
    const int lane = threadIdx.x & 31;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(a.queue + 1, 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total) break;
        const int g = base + lane;
        const int i = g / TPA, sub = g % TPA;
        const bool active = i < a.n_atoms;
        int zi = 0, cnt = 0;
        if (active) {
            zi = clamp_species(a.types[i], a.S);
            cnt = a.count[i];
        }
#if MTPGEN_HAS_PARTS
        if constexpr (PairgradMerged<T, TPA>::value) {
            pairgrad_merged<T, TPA>(a, i, sub, active, zi, cnt, cs, sadj);
            continue;
        }
#endif
        pairgrad_all<T, 0, NumSlices<T>::value, TPA>(a, i, sub, active, zi, cnt, cs, sadj);
    }
}

// ----------------------------------------------------------------------------------------------
// k_gather: forces and virial
// ----------------------------------------------------------------------------------------------
// running per-configuration sums of the gather: the virial in the working precision T (its
// per-pair terms are T already), the energy as a float pair in double-float arithmetic (about 44
// significant bits, so that E equals the double sum of the site energies, Eq. 2, to ~1e-13
// relative, with no double-precision arithmetic per atom); both reach the double outputs by atomics
template <class T>
__device__ __forceinline__ void flush_run(const EvalCtx<T>& a, int cfg, const T* run, double erun, bool want_e) {
    if (a.virial) {
#pragma unroll
        for (int k = 0; k < 9; ++k) atomicAdd(&a.virial[(size_t)cfg * 9 + k], (double)run[k]);
    }
    if (want_e) atomicAdd(&a.energy[cfg], erun);
}

template <class T>
struct GatherIn {
    Vec4<T> g;
    T rx, ry, rz;
    int rev, j;
};

template <class T, int TPA>
__global__ void __launch_bounds__(128, TPA >= 4 ? 8 : 1) k_gather(const EvalCtx<T> a) {
    pdl_enter();
    // float path with contraction parts: the site energies are the sums of the parts' shares
#if MTPGEN_HAS_PARTS
    constexpr bool kE = sizeof(T) == 4;
#else
    constexpr bool kE = false;
#endif
    const bool want_e = kE && a.energy != nullptr;
    constexpr int kWarps = 4;  // blockDim.x == 128
    __shared__ int s_cfg[kWarps];
    __shared__ T s_w[kWarps][9];
    __shared__ double s_e[kWarps];
    const size_t n = (size_t)a.n_atoms;
    const int stride = gridDim.x * blockDim.x;
    const int n_groups = ((a.n_atoms + 31) / 32) * 32;  // whole warps stay converged for the shuffles
    T Wrun[9];
    Df Erun = {0.f, 0.f};  // energy: an unevaluated float pair (error-free sums, no FP64 work)
#pragma unroll
    for (int k = 0; k < 9; ++k) Wrun[k] = T(0);
    int wcfg = -1;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n_groups * TPA; g += stride) {
        const int i = g / TPA, sub = g % TPA;
        const bool active = i < a.n_atoms;
        T F[3] = {T(0), T(0), T(0)};
        T W[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) W[k] = T(0);
        int cfg = -1;
        if (active) {
            cfg = a.cfg_of[i];
            const int cnt = a.count[i];
            if constexpr (TPA >= 4) {
                // few pairs per lane: the other warps hide the load latency
                for (int p = sub; p < cnt; p += TPA) {
                    const size_t idx = (size_t)p * n + i;
                    const Vec4<T> gv = a.g[idx];
                    const PairRec<T> pq = a.pr[idx];
                    const T g3[3] = {gv.x, gv.y, gv.z};
                    const T r[3] = {pq.x, pq.y, pq.z};
#pragma unroll
                    for (int u = 0; u < 3; ++u) {
                        F[u] += g3[u];
#pragma unroll
                        for (int v = 0; v < 3; ++v) W[3 * u + v] -= g3[u] * r[v];
                    }
                    const int q = a.rev[idx];
                    if (q >= 0) {
                        const Vec4<T> gr = a.g[(size_t)q * n + (pq.jz & 0xffffff)];
                        F[0] -= gr.x;
                        F[1] -= gr.y;
                        F[2] -= gr.z;
                    }
                }
            } else {
                // two-stage pipeline: the direct loads of pair p + 2 TPA and the reverse-pair load of
                // pair p + TPA are in flight while pair p is accumulated
                auto direct = [&](int p) {
                    GatherIn<T> d;
                    const size_t idx = (size_t)p * n + i;
                    d.g = a.g[idx];
                    const PairRec<T> pq = a.pr[idx];
                    d.rx = pq.x;
                    d.ry = pq.y;
                    d.rz = pq.z;
                    d.rev = a.rev[idx];
                    d.j = pq.jz & 0xffffff;
                    return d;
                };
                auto reverse = [&](const GatherIn<T>& d) {
                    return d.rev >= 0 ? a.g[(size_t)d.rev * n + d.j] : Vec4<T>{T(0), T(0), T(0), T(0)};
                };
                GatherIn<T> d0, d1;
                Vec4<T> r0{T(0), T(0), T(0), T(0)};
                if (sub < cnt) {
                    d0 = direct(sub);
                    r0 = reverse(d0);
                }
                if (sub + TPA < cnt) d1 = direct(sub + TPA);
                for (int p = sub; p < cnt; p += TPA) {
                    const GatherIn<T> cur = d0;
                    const Vec4<T> cr = r0;
                    if (p + TPA < cnt) {
                        d0 = d1;
                        r0 = reverse(d0);
                        if (p + 2 * TPA < cnt) d1 = direct(p + 2 * TPA);
                    }
                    const T g3[3] = {cur.g.x, cur.g.y, cur.g.z};
                    const T r[3] = {cur.rx, cur.ry, cur.rz};
    #pragma unroll
                    for (int u = 0; u < 3; ++u) {
                        F[u] += g3[u];
    #pragma unroll
                        for (int v = 0; v < 3; ++v) W[3 * u + v] -= g3[u] * r[v];
                    }
                    F[0] -= cr.x;
                    F[1] -= cr.y;
                    F[2] -= cr.z;
                }
            }
        }
        if (TPA > 1) {
#pragma unroll
            for (int o = 1; o < TPA; o <<= 1) {
#pragma unroll
                for (int u = 0; u < 3; ++u) F[u] += __shfl_xor_sync(0xffffffffu, F[u], o);
            }
        }
        if (active && sub == 0 && a.forces) {
            a.forces[3 * (size_t)i + 0] = (double)F[0];
            a.forces[3 * (size_t)i + 1] = (double)F[1];
            a.forces[3 * (size_t)i + 2] = (double)F[2];
        }
        float e_i = 0.f;
        if constexpr (kE) {
            if (active && sub == 0) {
                float e = 0.f;
#pragma unroll
                for (int p = 0; p < G::NPART_; ++p) e += a.epart[(size_t)p * n + i];
                if (a.site) a.site[i] = (double)e;
                e_i = e;
            }
        }
        if (active && (a.virial || want_e)) {
            if (cfg != wcfg) {
                if (wcfg >= 0) flush_run(a, wcfg, Wrun, (double)Erun.hi + (double)Erun.lo, want_e);
#pragma unroll
                for (int k = 0; k < 9; ++k) Wrun[k] = T(0);
                Erun = {0.f, 0.f};
                wcfg = cfg;
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) Wrun[k] += W[k];
            if (want_e) Erun = df_add(Erun, {e_i, 0.f});
        }
    }
    if (!a.virial && !want_e) return;
    // combine the running sums: a warp whose lanes all end in one configuration (lanes without atoms
    // hold zeros) sums them with shuffles, any other warp flushes lane by lane; then one thread per
    // component adds the warp sums, one double atomic per run of warps of equal configuration
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cmax = __reduce_max_sync(0xffffffffu, wcfg);
    const bool wuni = __all_sync(0xffffffffu, wcfg == cmax || wcfg < 0);
    if (wuni) {
        if (a.virial) {
#pragma unroll
            for (int k = 0; k < 9; ++k) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) Wrun[k] += __shfl_xor_sync(0xffffffffu, Wrun[k], o);
            }
        }
        if (want_e) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const Df other = {__shfl_xor_sync(0xffffffffu, Erun.hi, o), __shfl_xor_sync(0xffffffffu, Erun.lo, o)};
                Erun = df_add(Erun, other);
            }
        }
        if (lane < 9) {
            T v = Wrun[0];
#pragma unroll
            for (int k = 1; k < 9; ++k) v = lane == k ? Wrun[k] : v;
            s_w[warp][lane] = v;
        }
        if (lane == 9) s_e[warp] = (double)Erun.hi + (double)Erun.lo;
    } else if (wcfg >= 0) {
        flush_run(a, wcfg, Wrun, (double)Erun.hi + (double)Erun.lo, want_e);
    }
    if (lane == 0) s_cfg[warp] = wuni ? cmax : -1;  // -1: nothing left to add
    __syncthreads();
    if (threadIdx.x < 10) {
        const int k = threadIdx.x;
        const bool use = k < 9 ? a.virial != nullptr : want_e;
        double acc = 0.0;
        int cur = -1;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const int c = s_cfg[w];
            if (c < 0) continue;
            if (c != cur) {
                if (cur >= 0 && use) atomicAdd(k < 9 ? &a.virial[(size_t)cur * 9 + k] : &a.energy[cur], acc);
                acc = 0.0;
                cur = c;
            }
            acc += k < 9 ? (double)s_w[w][k] : s_e[w];
        }
        if (cur >= 0 && use) atomicAdd(k < 9 ? &a.virial[(size_t)cur * 9 + k] : &a.energy[cur], acc);
    }
}

// ----------------------------------------------------------------------------------------------
// launcher
// ----------------------------------------------------------------------------------------------
template <class T, int TPA>
int launch_pairs(const EvalCtx<T>& a, cudaStream_t st, int n_sm, bool moments) {
    const int threads = 128;
    const size_t cbytes = coef_bytes(a);
    const long work = (long)(((a.n_atoms + 31) / 32) * 32) * TPA;
    int blocks = (int)((work + threads - 1) / threads);
    const int max_blocks = n_sm * 16;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    if (moments) {
        static bool attr_m = false;
        if (!attr_m && cbytes > 48 * 1024) {  // 8 species with 16 radial functions in double
            cudaFuncSetAttribute(k_moments<T, TPA>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
            attr_m = true;
        }
        launch_pdl(k_moments<T, TPA>, blocks, threads, cbytes, st, a);
    } else {
        const size_t smem = ((cbytes + 15) & ~(size_t)15) + pairgrad_adj_bytes<T, TPA>();
        static bool attr_set = false;
        if (!attr_set && smem > 48 * 1024) {
            cudaFuncSetAttribute(k_pairgrad<T, TPA>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
            attr_set = true;
        }
        launch_pdl(k_pairgrad<T, TPA>, blocks, threads, smem, st, a);
    }
    return 1;
}

template <class T>
int launch_pairs_tpa(const EvalCtx<T>& a, cudaStream_t st, int n_sm, bool moments) {
    // the moment accumulation holds its sums in registers and takes tpa_m lanes per atom; the pair
    // gradients read dV/dM from shared memory and take the gather's tpa
    switch (moments ? a.tpa_m : a.tpa) {
        case 8: return launch_pairs<T, 8>(a, st, n_sm, moments);
        case 4: return launch_pairs<T, 4>(a, st, n_sm, moments);
        case 2: return launch_pairs<T, 2>(a, st, n_sm, moments);
        default: return launch_pairs<T, 1>(a, st, n_sm, moments);
    }
}

template <class T>
int eval_all(const EvalCtx<T>& a, cudaStream_t st, int n_sm, cudaEvent_t* marks, cudaEvent_t gather_after) {
    if (a.n_atoms == 0) return 0;
    int launches = 0;
    if (marks) record_mark(marks[kPhaseMoments], st);
    launches += launch_pairs_tpa<T>(a, st, n_sm, true);
    if (marks) record_mark(marks[kPhaseContract], st);
#if MTPGEN_HAS_PARTS
    if constexpr (sizeof(T) == 4) {
        const int threads = 128;
        // one warp per (part, tile) item and no grid-stride: the blocks resident at any time are a
        // window of consecutive part-major items, so an SM mostly runs one part's code (the parts are
        // long straight-line programs and their instruction fetch bounds the kernel otherwise)
        const long warps = (long)((a.n_atoms + 31) / 32) * G::NPART_;
        const int blocks = (int)((warps + 3) / 4);
        launch_pdl(k_contract_parts, blocks, threads, 0, st, a);
        ++launches;
        if (a.b_rows) {  // the caller provides per-atom rows whenever b rows are requested
            launch_pdl(k_brows<T>, a.n_cfg, 128, 0, st, a, a.cfg_off);
            ++launches;
        }
    } else
#endif
    {
        // atoms per warp: amortise each program word over several atoms while the per-warp working
        // set (2 A V values) stays small enough for at least two blocks per SM
        constexpr int A = (sizeof(T) * G::V_ * 2 * 4 * 8 <= 100 * 1024) ? 4
                        : (sizeof(T) * G::V_ * 2 * 2 * 8 <= 100 * 1024) ? 2 : 1;
        constexpr int threads = (sizeof(T) * G::V_ * 2 * A * 8 <= 100 * 1024) ? 256 : 128;
        const int wpb = threads / 32;
        const size_t smem = sizeof(T) * (size_t)G::V_ * (1 + 2 * A * wpb) + sizeof(float) * (a.n_weights + 4) + 64;
        if (smem > 200 * 1024) return -1000;  // not reachable for lev_max <= 20
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_contract<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr_set = true;
        }
        int per_sm = (int)((220 * 1024) / (smem + 1024));
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 8) per_sm = 8;
        int blocks = (a.n_atoms + wpb * A - 1) / (wpb * A);
        if (blocks > n_sm * per_sm) blocks = n_sm * per_sm;
        launch_pdl(k_contract<T, A>, blocks, threads, smem, st, a);
        ++launches;
    }
    if (marks) record_mark(marks[kPhasePairgrad], st);
    launches += launch_pairs_tpa<T>(a, st, n_sm, false);
    if (gather_after) cudaStreamWaitEvent(st, gather_after, 0);
    if (marks) record_mark(marks[kPhaseGather], st);
    {
        const int threads = 128;
        const long work = (long)(((a.n_atoms + 31) / 32) * 32) * a.tpa;
        int blocks = (int)((work + threads - 1) / threads);
        if (blocks > n_sm * 8) blocks = n_sm * 8;
        // after a wait on another stream's event the launch is an ordinary one
        auto go = [&](void (*k)(const EvalCtx<T>)) {
            if (gather_after)
                k<<<blocks, threads, 0, st>>>(a);
            else
                launch_pdl(k, blocks, threads, 0, st, a);
        };
        switch (a.tpa) {
            case 8: go(k_gather<T, 8>); break;
            case 4: go(k_gather<T, 4>); break;
            case 2: go(k_gather<T, 2>); break;
            default: go(k_gather<T, 1>); break;
        }
        ++launches;
    }
    if (marks) record_mark(marks[kPhases], st);
    return launches;
}

int eval_f32(const EvalCtx<float>& a, cudaStream_t st, int n_sm, cudaEvent_t* marks, cudaEvent_t gather_after) {
    return eval_all<float>(a, st, n_sm, marks, gather_after);
}
int eval_f64(const EvalCtx<double>& a, cudaStream_t st, int n_sm, cudaEvent_t* marks, cudaEvent_t gather_after) {
    return eval_all<double>(a, st, n_sm, marks, gather_after);
}


// ----------------------------------------------------------------------------------------------
// Training-loss gradient (Sec. 2.2, Eqs. 7, 11, 12).  With e_k = 2 s_e w_e dE_k, D_i = 2 s_f w_f dF_i
// and eps_k = 2 s_s w_s dW_k, the force and stress terms equal -dG/dtheta for
// G = sum_pairs g_ij . u_ij, u_ij = (D_j - D_i) + eps_k r_ij (g_ij = dV_i/dr_ij), so
//   dL/dxi_a = sum_i (e_k B_a(n_i) - dB_a/dt),
//   dL/dc    = sum_pairs (e_k Q_b P_mu - Q'_b (r-hat . u) P_mu - Q_b dP_mu/dt),
// with P_mu = sum_m dV/dM[mu,m] mono_m and d/dt the derivative along u (forward mode): the moments'
// tangent comes from k_tmom, the programs run again on (value, tangent) pairs.
// ----------------------------------------------------------------------------------------------
template <class T>
__global__ void k_resid_atoms(EvalCtx<T> a, LossArgs L, T* D) {
    __shared__ double s_l[128];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n_atoms; i += gridDim.x * blockDim.x) {
        const int k = L.cfg_of[i];
        double se, sf, ss;
        loss_scales(L.scaling, (double)(L.cfg_off[k + 1] - L.cfg_off[k]), &se, &sf, &ss);
        double q = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double d = L.forces[3 * (size_t)i + c] - L.f_ref[3 * (size_t)i + c];
            D[3 * (size_t)i + c] = (T)(2.0 * sf * L.wf * d);
            q += d * d;
        }
        acc += sf * L.wf * q;
    }
    s_l[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s_l[threadIdx.x] += s_l[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(L.loss, s_l[0]);
}

template <class T>
__global__ void k_resid_cfgs(LossArgs L, T* eps) {
    __shared__ double s_l[128];
    double acc = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L.n_cfg; k += gridDim.x * blockDim.x) {
        double se, sf, ss;
        loss_scales(L.scaling, (double)(L.cfg_off[k + 1] - L.cfg_off[k]), &se, &sf, &ss);
        const double de = L.energy[k] - L.e_ref[k];
        L.gew[k] = 2.0 * se * L.we * de;
        double q = 0.0;
        for (int c = 0; c < 9; ++c) {
            const double dw = L.virial[9 * (size_t)k + c] - L.w_ref[9 * (size_t)k + c];
            eps[9 * (size_t)k + c] = (T)(2.0 * ss * L.ws * dw);
            q += dw * dw;
        }
        acc += se * L.we * de * de + ss * L.ws * q;
    }
    s_l[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s_l[threadIdx.x] += s_l[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(L.loss, s_l[0]);
}

// pair displacement direction u_ij = (D_j - D_i) + eps_k r_ij
template <class T>
__device__ __forceinline__ void pair_u(const EvalCtx<T>& a, const T* Di, const T* E, int j, T x, T y, T z, T& ux,
                                       T& uy, T& uz) {
    ux = (a.gD[3 * (size_t)j] - Di[0]) + (E[0] * x + E[1] * y + E[2] * z);
    uy = (a.gD[3 * (size_t)j + 1] - Di[1]) + (E[3] * x + E[4] * y + E[5] * z);
    uz = (a.gD[3 * (size_t)j + 2] - Di[2]) + (E[6] * x + E[7] * y + E[8] * z);
}

template <class T, int S, int TPA>
__device__ __forceinline__ void tmom_slice(const EvalCtx<T>& a, int i, int sub, bool active, int zi, int cnt,
                                           const T* cs, const T* Di, const T* E) {
    using SL = typename SliceSel<T, S>::type;
    T acc[SL::SIZE];
#pragma unroll
    for (int t = 0; t < SL::SIZE; ++t) acc[t] = T(0);
    const size_t n = (size_t)a.n_atoms;
    if (active) {
        const int csz = coef_row(a);
        for (int p = sub; p < cnt; p += TPA) {
            const size_t idx = (size_t)p * n + i;
            const PairRec<T> pq = a.pr[idx];
            const int j = pq.jz & 0xffffff, zj = pq.jz >> 24;
            const T x = pq.x, y = pq.y, z = pq.z;
            const T r = my_sqrt(x * x + y * y + z * z);
            T f[G::NMU_], df[G::NMU_];
            radial<T, true>(r, cs + (zi * a.S + zj) * csz, a.NQ, a.rmin, a.rcut, a.inv_span, f, df);
            T ux, uy, uz;
            pair_u(a, Di, E, j, x, y, z, ux, uy, uz);
            const T rdu = (x * ux + y * uy + z * uz) / r;
            SL::template tmom<T>(x, y, z, f, df, rdu, ux, uy, uz, acc);
        }
    }
    if (TPA > 1) {
#pragma unroll
        for (int t = 0; t < SL::SIZE; ++t) {
#pragma unroll
            for (int o = 1; o < TPA; o <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
        }
    }
    if (active) {
        T* dst = a.momt + (size_t)(i >> 5) * G::C_ * 32 + (i & 31);
#pragma unroll
        for (int t = 0; t < SL::SIZE; ++t)
            if (t % TPA == sub) dst[(size_t)(SL::BEGIN + t) * 32] = acc[t];
    }
}

template <class T, int S, int NS, int TPA>
__device__ __forceinline__ void tmom_all(const EvalCtx<T>& a, int i, int sub, bool active, int zi, int cnt,
                                         const T* cs, const T* Di, const T* E) {
    if constexpr (S < NS) {
        tmom_slice<T, S, TPA>(a, i, sub, active, zi, cnt, cs, Di, E);
        tmom_all<T, S + 1, NS, TPA>(a, i, sub, active, zi, cnt, cs, Di, E);
    }
}

template <class T, int TPA>
__global__ void __launch_bounds__(128) k_tmom(const EvalCtx<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* cs = reinterpret_cast<T*>(smem_raw);
    load_c(a, cs);
    const int stride = gridDim.x * blockDim.x;
    const int n_groups = ((a.n_atoms + 31) / 32) * 32;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n_groups * TPA; g += stride) {
        const int i = g / TPA, sub = g % TPA;
        const bool active = i < a.n_atoms;
        int zi = 0, cnt = 0;
        T Di[3] = {T(0), T(0), T(0)}, E[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) E[q] = T(0);
        if (active) {
            zi = clamp_species(a.types[i], a.S);
            cnt = a.count[i];
            for (int q = 0; q < 3; ++q) Di[q] = a.gD[3 * (size_t)i + q];
            const int k = a.cfg_of[i];
            for (int q = 0; q < 9; ++q) E[q] = a.geps[9 * (size_t)k + q];
        }
        tmom_all<T, 0, NumSlices<T>::value, TPA>(a, i, sub, active, zi, cnt, cs, Di, E);
    }
}

// forward and adjoint programs on (value, tangent) pairs, warp per atom
template <class T, bool ADJ>
__device__ __forceinline__ void run_program_dual(const unsigned long long* __restrict__ ops,
                                                 const int* __restrict__ layer_end, int layers, const float* sw,
                                                 T* val, T* tan, T* adj, T* adt, int lane) {
    int row = 0;
    for (int l = 0; l < layers; ++l) {
        const int end = layer_end[l];
        T acc = T(0), acct = T(0);
        for (; row < end; ++row) {
            const unsigned long long op = ops[row * 32 + lane];
            const unsigned fl = (unsigned)(op >> 48) & 7u;
            if (fl & 4u) continue;
            const int i = (int)(op & 0xffffu), j = (int)((op >> 16) & 0xffffu), k = (int)((op >> 32) & 0xffffu);
            const T w = (T)sw[op >> 51];
            if (ADJ) {
                if (fl & 1u) {
                    acc = adj[k];
                    acct = adt[k];
                }
                acc += w * val[i] * adj[j];
                acct += w * (tan[i] * adj[j] + val[i] * adt[j]);
                if (fl & 2u) {
                    adj[k] = acc;
                    adt[k] = acct;
                }
            } else {
                if (fl & 1u) {
                    acc = T(0);
                    acct = T(0);
                }
                acc += w * val[i] * val[j];
                acct += w * (tan[i] * val[j] + val[i] * tan[j]);
                if (fl & 2u) {
                    val[k] = acc;
                    tan[k] = acct;
                }
            }
        }
        __syncwarp();
    }
}

#if MTPGEN_HAS_PARTS
// Tangent contraction of the loss gradient (float), split into NDPART generated parts like the
// forward contraction: warp w runs part w / n_tiles for the 32 atoms of tile w % n_tiles.  Each part
// writes dV/dM and its tangent for its moments to dual slots and its basis functions' shares of
// dL/dxi (summed over the tile's atoms) to dxt[tile].
__global__ void __launch_bounds__(128) k_contract_tan_parts(const EvalCtx<float> a) {
    const int lane = threadIdx.x & 31;
    const int n_tiles = (a.n_atoms + 31) >> 5;
    const int total = n_tiles * G::NDPART_;
    const size_t half = (size_t)n_tiles * G::NDSLOT_ * 32;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += (gridDim.x * blockDim.x) >> 5) {
        const int part = w / n_tiles, tile = w - part * n_tiles;
        const int i = tile * 32 + lane;
        const bool act = i < a.n_atoms;
        const double ek = act ? a.gew[a.cfg_of[i]] : 0.0;
        const size_t mo = (size_t)tile * G::C_ * 32 + lane;
        const size_t so = (size_t)tile * G::NDSLOT_ * 32 + lane;
        ::MTP_GEN_NS::dual_part(part, a.mom + mo, a.momt + mo, a.dslots + so, a.dslots + half + so, a.xi, ek, act,
                                lane == 0, a.dxt + (size_t)tile * G::M_);
    }
}

// dV/dM and its tangent = sums of their dual slots (slot order), one warp per (tile, component)
__global__ void __launch_bounds__(128) k_dual_sum(const EvalCtx<float> a) {
    constexpr int C = G::C_;
    const int lane = threadIdx.x & 31;
    const int n_tiles = (a.n_atoms + 31) >> 5;
    const size_t half = (size_t)n_tiles * G::NDSLOT_ * 32;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_tiles * C; w += warps) {
        const int tile = w / C, c = w - tile * C;
        const float* sl = a.dslots + (size_t)tile * G::NDSLOT_ * 32 + lane;
        const int s0 = ::MTP_GEN_NS::dslot_begin[c], s1 = ::MTP_GEN_NS::dslot_begin[c + 1];
        float va = 0.f, vt = 0.f;
        for (int s = s0; s < s1; ++s) {
            va += sl[s * 32];
            vt += sl[half + s * 32];
        }
        const size_t q = ((size_t)tile * C + c) * 32 + lane;
        a.adjm[q] = va;
        a.adjmt[q] = vt;
    }
}

// dL/dxi += sum over tiles of dxt (one block per basis function, fixed reduction order)
__global__ void __launch_bounds__(128) k_dx_sum(const EvalCtx<float> a) {
    __shared__ double s[128];
    const int alpha = blockIdx.x;
    const int n_tiles = (a.n_atoms + 31) >> 5;
    double acc = 0.0;
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) acc += a.dxt[(size_t)t * G::M_ + alpha];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&a.dxi[alpha], s[0]);
}
#endif

template <class T>
__global__ void __launch_bounds__(128) k_contract_tan(const EvalCtx<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int V = G::V_, C = G::C_, M = G::M_;
    constexpr int MB = (M + 31) / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    T* seed = reinterpret_cast<T*>(smem_raw);
    float* sw = reinterpret_cast<float*>(seed + V);
    T* val = reinterpret_cast<T*>(sw + ((a.n_weights + 3) & ~3)) + (size_t)warp * 4 * V;
    T* tan = val + V;
    T* adj = tan + V;
    T* adt = adj + V;
    for (int v = threadIdx.x; v < V; v += blockDim.x) seed[v] = a.seed[v];
    for (int v = threadIdx.x; v < a.n_weights; v += blockDim.x) sw[v] = a.weights[v];
    __syncthreads();
    double dx[MB];
#pragma unroll
    for (int t = 0; t < MB; ++t) dx[t] = 0.0;
    for (int i = blockIdx.x * wpb + warp; i < a.n_atoms; i += gridDim.x * wpb) {
        const size_t tb = (size_t)(i >> 5) * C * 32 + (i & 31);
        for (int c = lane; c < C; c += 32) {
            val[c] = a.mom[tb + (size_t)c * 32];
            tan[c] = a.momt[tb + (size_t)c * 32];
        }
        __syncwarp();
        run_program_dual<T, false>(a.fwd_ops, a.fwd_layer_end, a.fwd_layers, sw, val, tan, adj, adt, lane);
        const double ek = a.gew[a.cfg_of[i]];
#pragma unroll
        for (int t = 0; t < MB; ++t) {
            const int al = lane + 32 * t;
            if (al < M) {
                const int v = a.basis_value[al];
                dx[t] += ek * (double)val[v] - (double)tan[v];
            }
        }
        for (int v = lane; v < V; v += 32) {
            adj[v] = seed[v];
            adt[v] = T(0);
        }
        __syncwarp();
        run_program_dual<T, true>(a.adj_ops, a.adj_layer_end, a.adj_layers, sw, val, tan, adj, adt, lane);
        for (int c = lane; c < C; c += 32) {
            a.adjm[tb + (size_t)c * 32] = adj[c];
            a.adjmt[tb + (size_t)c * 32] = adt[c];
        }
        __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < MB; ++t)
        if (lane + 32 * t < M) atomicAdd(&a.dxi[lane + 32 * t], dx[t]);
}

template <class T, int S, int NS>
__device__ __forceinline__ void pdot_all(const T* adjp, const T* adjtp, T x, T y, T z, T ux, T uy, T uz, T* P,
                                         T* Pd) {
    if constexpr (S < NS) {
        using SL = typename SliceSel<T, S>::type;
        SL::template pdot<T>(x, y, z, adjp + (size_t)SL::BEGIN * 32, adjtp + (size_t)SL::BEGIN * 32, ux, uy, uz, P,
                             Pd);
        pdot_all<T, S + 1, NS>(adjp, adjtp, x, y, z, ux, uy, uz, P, Pd);
    }
}

// dL/dc: thread group per atom, one pass per neighbour species (register accumulators, when the
// radial basis size NQC is a compile-time constant; 0 = any size), then shared-memory and global
// double atomics
template <class T, int TPA, int NQC>
__global__ void __launch_bounds__(128) k_dc(const EvalCtx<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NMU = G::NMU_;
    const int nc = a.S * a.S * NMU * a.NQ;
    double* dcs = reinterpret_cast<double*>(smem_raw);
    for (int k = threadIdx.x; k < nc; k += blockDim.x) dcs[k] = 0.0;
    __syncthreads();
    const size_t n = (size_t)a.n_atoms;
    const int NQ = NQC ? NQC : a.NQ;
    constexpr int NQM = NQC ? NQC : kMaxRadial;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.n_atoms * TPA; g += gridDim.x * blockDim.x) {
        const int i = g / TPA, sub = g % TPA;
        const int zi = clamp_species(a.types[i], a.S);
        const int cnt = a.count[i];
        const int k = a.cfg_of[i];
        const T ek = (T)a.gew[k];
        T Di[3], E[9];
        for (int q = 0; q < 3; ++q) Di[q] = a.gD[3 * (size_t)i + q];
        for (int q = 0; q < 9; ++q) E[q] = a.geps[9 * (size_t)k + q];
        const size_t tb = (size_t)(i >> 5) * G::C_ * 32 + (i & 31);
        for (int zp = 0; zp < a.S; ++zp) {
            T acc[NMU][NQM];
#pragma unroll
            for (int mu = 0; mu < NMU; ++mu)
#pragma unroll
                for (int b = 0; b < NQM; ++b) acc[mu][b] = T(0);
            bool any = false;
            for (int p = sub; p < cnt; p += TPA) {
                const size_t idx = (size_t)p * n + i;
                const PairRec<T> pq = a.pr[idx];
                if ((pq.jz >> 24) != zp) continue;
                any = true;
                const int j = pq.jz & 0xffffff;
                const T x = pq.x, y = pq.y, z = pq.z;
                const T r = my_sqrt(x * x + y * y + z * z);
                T ux, uy, uz;
                pair_u(a, Di, E, j, x, y, z, ux, uy, uz);
                const T rdu = (x * ux + y * uy + z * uz) / r;
                T P[NMU], Pd[NMU];
#pragma unroll
                for (int mu = 0; mu < NMU; ++mu) P[mu] = Pd[mu] = T(0);
                pdot_all<T, 0, NumSlices<T>::value>(a.adjm + tb, a.adjmt + tb, x, y, z, ux, uy, uz, P, Pd);
                // Q_b = T_b(x) u^2 and dQ_b/dr (Eq. 4)
                const T xx = (T(2) * r - a.rmin - a.rcut) * a.inv_span;
                const T uu = r < a.rcut ? a.rcut - r : T(0);  // Q_b = 0 beyond the cutoff (Eq. 4)
                T t0 = T(1), t1 = xx, d0 = T(0), d1 = T(1);
#pragma unroll
                for (int b = 0; b < NQM; ++b) {
                    if (!NQC && b >= NQ) break;
                    T tb_, db_;
                    if (b == 0) {
                        tb_ = t0;
                        db_ = d0;
                    } else if (b == 1) {
                        tb_ = t1;
                        db_ = d1;
                    } else {
                        const T t2 = T(2) * xx * t1 - t0, d2 = T(2) * t1 + T(2) * xx * d1 - d0;
                        t0 = t1;
                        t1 = t2;
                        d0 = d1;
                        d1 = d2;
                        tb_ = t2;
                        db_ = d2;
                    }
                    const T Q = tb_ * uu * uu;
                    const T dQ = db_ * (T(2) * a.inv_span) * uu * uu - T(2) * tb_ * uu;
#pragma unroll
                    for (int mu = 0; mu < NMU; ++mu) acc[mu][b] += ek * Q * P[mu] - dQ * rdu * P[mu] - Q * Pd[mu];
                }
            }
            if (any) {
                // the loss gradient sums over the batch (shared memory first); Jacobian rows go to
                // their configuration's row directly
                double* dst = (a.dc_rows ? a.dc_rows + (size_t)k * nc : dcs) + (size_t)((zi * a.S + zp) * NMU) * NQ;
#pragma unroll
                for (int mu = 0; mu < NMU; ++mu)
#pragma unroll
                    for (int b = 0; b < NQM; ++b)
                        if (NQC || b < NQ) atomicAdd(&dst[mu * NQ + b], (double)acc[mu][b]);
            }
        }
    }
    __syncthreads();
    if (!a.dc_rows)
        for (int q = threadIdx.x; q < nc; q += blockDim.x)
            if (dcs[q] != 0.0) atomicAdd(&a.dc[q], dcs[q]);
}

template <class T, int TPA>
int launch_grad_pairs(EvalCtx<T>& a, cudaStream_t st, int n_sm) {
    const int threads = 128;
    const long work = (long)(((a.n_atoms + 31) / 32) * 32) * TPA;
    int blocks = (int)((work + threads - 1) / threads);
    if (blocks > n_sm * 16) blocks = n_sm * 16;
    if (blocks < 1) blocks = 1;
    const size_t cbytes = coef_bytes(a);
    static bool attr_t = false;
    if (!attr_t && cbytes > 48 * 1024) {
        cudaFuncSetAttribute(k_tmom<T, TPA>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        attr_t = true;
    }
    k_tmom<T, TPA><<<blocks, threads, cbytes, st>>>(a);
    return 1;
}

template <class T>
int grad_all(EvalCtx<T>& a, const LossArgs& L, cudaStream_t st, int n_sm) {
    int launches = 0;
    T* D = const_cast<T*>(a.gD);
    T* eps = const_cast<T*>(a.geps);
    if (!L.jacobian) {
        k_resid_atoms<T><<<min((a.n_atoms + 127) / 128 + 1, n_sm * 8), 128, 0, st>>>(a, L, D);
        k_resid_cfgs<T><<<min((a.n_cfg + 127) / 128 + 1, n_sm * 8), 128, 0, st>>>(L, eps);
        launches += 2;
    }
    if (a.n_atoms == 0 || L.loss_only) return launches;
    switch (a.tpa) {
        case 8: launches += launch_grad_pairs<T, 8>(a, st, n_sm); break;
        case 4: launches += launch_grad_pairs<T, 4>(a, st, n_sm); break;
        case 2: launches += launch_grad_pairs<T, 2>(a, st, n_sm); break;
        default: launches += launch_grad_pairs<T, 1>(a, st, n_sm); break;
    }
#if MTPGEN_HAS_PARTS
    if constexpr (sizeof(T) == 4) {
        const int n_tiles = (a.n_atoms + 31) / 32;
        const int blocks = (int)(((long)n_tiles * G::NDPART_ + 3) / 4);  // as for k_contract_parts
        k_contract_tan_parts<<<blocks, 128, 0, st>>>(a);
        int sblocks = (int)(((long)n_tiles * G::C_ + 3) / 4);
        if (sblocks > n_sm * 32) sblocks = n_sm * 32;
        k_dual_sum<<<sblocks, 128, 0, st>>>(a);
        k_dx_sum<<<G::M_, 128, 0, st>>>(a);
        launches += 3;
    } else
#endif
    {
        const int threads = 128, wpb = 4;
        const size_t smem = sizeof(T) * (size_t)G::V_ * (1 + 4 * wpb) + sizeof(float) * (a.n_weights + 4) + 64;
        if (smem > 200 * 1024) return -1000;
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_contract_tan<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr_set = true;
        }
        int per_sm = (int)((220 * 1024) / (smem + 1024));
        if (per_sm < 1) per_sm = 1;
        int blocks = (a.n_atoms + wpb - 1) / wpb;
        if (blocks > n_sm * per_sm) blocks = n_sm * per_sm;
        k_contract_tan<T><<<blocks, threads, smem, st>>>(a);
        ++launches;
    }
    {
        const int threads = 128;
        const size_t smem = sizeof(double) * (size_t)a.S * a.S * G::NMU_ * a.NQ;
        int blocks = (a.n_atoms + threads - 1) / threads;
        if (blocks > n_sm * 8) blocks = n_sm * 8;
        if (a.NQ == 8)
            k_dc<T, 1, 8><<<blocks, threads, smem, st>>>(a);
        else
            k_dc<T, 1, 0><<<blocks, threads, smem, st>>>(a);
        ++launches;
    }
    return launches;
}

int grad_f32(EvalCtx<float>& a, const LossArgs& L, cudaStream_t st, int n_sm) { return grad_all<float>(a, L, st, n_sm); }
int grad_f64(EvalCtx<double>& a, const LossArgs& L, cudaStream_t st, int n_sm) { return grad_all<double>(a, L, st, n_sm); }

}  // namespace MTP_GEN_NS

const LevelOps* MTP_LEVEL_FN() {
    namespace g = ::MTP_GEN_NS;
    static const LevelOps ops = {
        g::L, g::C, g::V, g::M, g::NMU, g::NUMAX,
        g::level_table, g::LEVEL_TABLE_LEN, g::basis_value,
        g::fwd_ops, g::fwd_layer_rows, g::FWD_ROWS, g::FWD_LAYERS,
        g::adj_ops, g::adj_layer_rows, g::ADJ_ROWS, g::ADJ_LAYERS, g::weights, g::NWEIGHTS,
        g::PROGRAM_OPS, g::FLOP_PAIR_MOMENTS, g::FLOP_PAIR_ADJOINT, g::FLOP_ATOM_PROGRAM,
        g::Traits::NPART_, g::Traits::NSLOT_, g::Traits::NDPART_, g::Traits::NDSLOT_,
        &MTP_GEN_NS::eval_f32, &MTP_GEN_NS::eval_f64, &MTP_GEN_NS::grad_f32, &MTP_GEN_NS::grad_f64};
    return &ops;
}

}  // namespace mtp
