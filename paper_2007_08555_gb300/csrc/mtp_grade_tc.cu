// Extrapolation grade of Sec. 2.3 on the tensor cores: gamma_r = max_j |(b_r A^-1)_j| for many rows
// b_r (per-configuration or per-atom basis rows), with tcgen05 BF16 MMAs accumulating in FP32 in TMEM.
//
// The product is ill-conditioned (cond(A D) reaches 1e13 for real active sets, and c = b A^-1 is
// then a small difference of large terms), so plain BF16/TF32 inputs would lose every digit of c.
// It is computed as an exact integer product of digit expansions instead (the error-free splitting
// of Ozaki et al., 2012, with base-2^7 digits small enough for BF16):
//   1. column scaling by powers of two: b' = b D, G = (A D)^-1 = D^-1 A^-1, D_k = 2^e_k so that the
//      columns of A D have maxima in [1/2, 1) (c = b' G exactly, and the scaling itself is exact);
//   2. each row of b' is rounded to T_r,k = b'_rk 2^(56 - E_r) (an integer, |T| < 2^55, E_r from the
//      row's largest exponent), each column of G to U_k,j = G_kj 2^(56 - F_j), and both integers are
//      written as 8 base-128 digits q_s, p_t (balanced, |digit| <= 65: exact in BF16);
//   3. for every digit pair (s, t) with s + t <= 9 the tensor cores form sum_k q_s,k p_t,k; pairs with
//      the same g = s + t share one FP32 accumulator (8 groups, 8 x 64 TMEM columns).  Each group sum
//      is an integer below 8 x 460 x 65^2 < 2^24, so the FP32 accumulation is exact;
//   4. the epilogue combines the groups exactly in 64-bit integers,
//      sum_k T_r,k U_k,j ~ 2^49 (sum_g A_g 128^(9-g)),  c_rj = 2^(E_r + F_j - 63) (sum_g A_g 128^(9-g)),
//      rounds once to float and keeps the row maximum of |c|.
// Error: the rounding of b' and G to 56-bit grids and the dropped pairs (s + t >= 10) are each below
// ~1e-15 of 2^(E_r + F_j) (the scales of the row and the column), comparable to a double-precision
// product; the final rounding to float adds 2^-24 relative to gamma.  Rows holding NaN or inf get
// gamma = +inf.
//
// Layout (shared memory, canonical K-major without swizzle): a plane of R rows x 64 k of BF16 is
// made of 8 x 8 core matrices of 8 rows x 16 bytes; element (r, k) sits at
// (r / 8) * 1024 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2 bytes (k groups 128 bytes apart: the
// descriptor's leading byte offset; row groups 1024 bytes apart: its stride byte offset).
//
// One persistent CTA per SM (256 threads, 195 KB of shared memory, all 512 TMEM columns) walks over
// tiles of 128 rows x 64 output columns; per 64-wide K chunk: the column digits of G are copied from
// global memory by the bulk-copy engine (cp.async.bulk, prepared once per active set), the threads
// write the row digits, one thread issues the 36 x 4 MMAs and commits them to an mbarrier.  Every
// wait on an mbarrier gives up after ~2 s, sets the error word and leaves the kernel.
#include <cuda_runtime.h>
#include <stdint.h>
#include "mtp_common.cuh"
#include "mtp_internal.h"

namespace mtp {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcRows = 128;                   // M of the MMA (rows of b per tile)
constexpr int kTcCols = 64;                    // N of the MMA (output columns per tile)
constexpr int kTcK = 64;                       // K per chunk
constexpr int kDigits = 8;                     // base-128 digits per operand
constexpr int kGroups = 8;                     // g = s + t = 2 .. 9
constexpr int kPlaneA = kTcRows * kTcK * 2;    // 16 KB
constexpr int kPlaneB = kTcCols * kTcK * 2;    // 8 KB
constexpr int kSmA = 0;
constexpr int kSmB = kSmA + kDigits * kPlaneA;             // 128 KB of row digits
constexpr int kSmMisc = kSmB + kDigits * kPlaneB;          // 64 KB of column digits
constexpr int kMaxK = 512;                                 // K padded to whole chunks
constexpr int kMaxM = 480;  // exact FP32 group sums need 8 pairs x m x 65 x 64 < 2^24 (lev_max 20: m = 460)
constexpr int kSmEk = kSmMisc + 64;                        // int [kMaxK]
constexpr int kSmErow = kSmEk + 4 * kMaxK;                 // int [128]
constexpr int kSmBad = kSmErow + 4 * kTcRows;              // int [128]
constexpr int kSmScale = kSmBad + 4 * kTcRows;             // float [64]
constexpr int kSmFlag = kSmScale + 4 * kTcCols;            // int
constexpr int kSmTotal = kSmFlag + 16;
constexpr int kSmAlloc = kSmTotal + 1024;                  // room to align the base to 1 KB
constexpr long long kWaitNs = 2000000000ll;                // give up on an mbarrier after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// shared-memory matrix descriptor: canonical K-major layout without swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);           // start address
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;     // leading byte offset: next 8 k
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;    // stride byte offset: next 8 rows
    d |= (uint64_t)1 << 46;                           // descriptor version of this architecture
    return d;                                         // base offset 0, no swizzle
}

// instruction descriptor, kind::f16: D in F32, A and B in BF16, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcCols >> 3) << 17) |
                            ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Wait for the phase with the given parity; false after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((long long)(global_ns() - t0) > kWaitNs) return false;
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

// Byte offset of element (r, k) in a plane (canonical K-major, no swizzle).
__host__ __device__ __forceinline__ int plane_off(int r, int k) {
    return (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// round(x 2^shift) for |x 2^shift| < 2^55 (the caller's choice of shift): an integer from the bits
// of x; zeros, subnormals, infinities and NaN give 0 (non-finite rows are flagged separately).
__device__ __forceinline__ long long fixed_point(double x, int shift) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((u >> 52) & 0x7ffu);
    if (ex == 0 || ex == 0x7ff) return 0;
    const long long mant = (long long)((u & 0xFFFFFFFFFFFFFull) | (1ull << 52));
    const int sh = ex - 1075 + shift;  // x = mant 2^(ex - 1075)
    long long t;
    if (sh >= 0)
        t = mant << (sh < 10 ? sh : 10);
    else if (sh > -60)
        t = (mant + (1ll << (-sh - 1))) >> (-sh);
    else
        t = 0;
    return (u >> 63) ? -t : t;
}

// unbiased exponent e with 2^e <= |x| < 2^(e+1), or INT_MIN / 2 for zero and subnormals
__device__ __forceinline__ int exponent_of(double x) {
    const int ex = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffu);
    return ex == 0 ? -(1 << 29) : ex - 1023;
}

// Eight base-128 digits of T (|T| < 2^55), most significant first; digits 2..8 balanced in
// [-64, 63], the first takes what remains (|q0| <= 65).  32-bit arithmetic on the two halves.
__device__ __forceinline__ void base128_digits(long long T, int* q) {
    int lo = (int)(T & ((1ll << 28) - 1));  // [0, 2^28)
    int hi = (int)(T >> 28);                // floor
#pragma unroll
    for (int s = 7; s >= 4; --s) {
        const int d = ((lo + 64) & 127) - 64;
        q[s] = d;
        lo = (lo - d) >> 7;
    }
    hi += lo;  // carry 0 or 1
#pragma unroll
    for (int s = 3; s >= 1; --s) {
        const int d = ((hi + 64) & 127) - 64;
        q[s] = d;
        hi = (hi - d) >> 7;
    }
    q[0] = hi;
}

// BF16 bits of a small integer (|d| < 2^8: exact)
__device__ __forceinline__ uint32_t bf16_bits(int d) {
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;  // exact for |d| < 2^22
    return __float_as_uint(f) >> 16;
}

// ------------------------------------------------------------------------------------------------
// Preparation once per active set: column exponents e_k of D, column scales F_j of G = (A D)^-1 and
// the digit planes of G in the layout of the MMA's B operand:
//   digits[((ct * n_kc + kc) * 8 + t) * 4096 + plane_off(j % 64, k % 64) / 2] = digit t of G_kj.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_grade_tc_prep(int m, const double* A, const double* Ai, uint16_t* digits,
                                                       int* ecol, float* cscale, int n_ct, int n_kc) {
    __shared__ int s_e[kMaxK];
    const int mpad = n_ct * kTcCols;
    // D_k = 2^e_k with max_r |A_rk| 2^e_k in [1/2, 1)
    for (int k = threadIdx.x; k < kMaxK; k += blockDim.x) {
        int e = 0;
        if (k < m) {
            int mx = -(1 << 29);
            for (int r = 0; r < m; ++r) mx = max(mx, exponent_of(A[(size_t)r * m + k]));
            e = mx > -(1 << 28) ? -(mx + 1) : 0;
        }
        s_e[k] = e;
        if (k < mpad) ecol[k] = e;
    }
    __syncthreads();
    // G_kj = Ai_kj 2^(-e_k); F_j from the column's largest exponent (|G_kj| < 2^(F_j - 1))
    for (int j = threadIdx.x; j < mpad; j += blockDim.x) {
        int F = 0;
        if (j < m) {
            int mx = -(1 << 29);
            for (int k = 0; k < m; ++k) mx = max(mx, exponent_of(Ai[(size_t)k * m + j]) - s_e[k]);
            F = mx > -(1 << 28) ? mx + 2 : 0;
        }
        // 2^(F - 63); a column whose entries are all below 2^-60 contributes nothing measurable
        cscale[j] = j >= m || F <= -60 ? 0.f : (F >= 120 ? (float)INFINITY : __int_as_float((F - 63 + 127) << 23));
        const int ct = j / kTcCols, jj = j % kTcCols;
        for (int k = 0; k < n_kc * kTcK; ++k) {
            int q[kDigits] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (j < m && k < m) base128_digits(fixed_point(Ai[(size_t)k * m + j], 56 - F - s_e[k]), q);
            const int kc = k / kTcK, kk = k % kTcK;
            const size_t base = ((size_t)(ct * n_kc + kc) * kDigits) * (kPlaneB / 2) + plane_off(jj, kk) / 2;
#pragma unroll
            for (int t = 0; t < kDigits; ++t) digits[base + (size_t)t * (kPlaneB / 2)] = (uint16_t)bf16_bits(q[t]);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// The grade kernel.
// ------------------------------------------------------------------------------------------------
struct TcArgs {
    int n, m, ldb;
    int n_ct, n_kc, n_tiles;
    const double* B;
    const uint16_t* digits;
    const int* ecol;
    const float* cscale;
    unsigned long long* gbits;
    int* err;
};

__global__ void __launch_bounds__(kTcThreads, 1) k_grade_tc(const TcArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kSmMisc);  // [0] MMAs done, [1] column digits landed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kSmMisc + 16);
    int* s_ek = reinterpret_cast<int*>(sm + kSmEk);
    int* s_erow = reinterpret_cast<int*>(sm + kSmErow);
    int* s_bad = reinterpret_cast<int*>(sm + kSmBad);
    float* s_scale = reinterpret_cast<float*>(sm + kSmScale);
    int* s_flag = reinterpret_cast<int*>(sm + kSmFlag);
    const uint32_t bar_mma = smem_u32(&bars[0]), bar_cp = smem_u32(&bars[1]);
    const uint32_t sA = smem_u32(sm + kSmA), sB = smem_u32(sm + kSmB);

    if (tid == 0) {
        mbar_init(bar_mma, 1);
        mbar_init(bar_cp, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_flag = 0;
    }
    for (int k = tid; k < kMaxK; k += kTcThreads) s_ek[k] = k < a.n_kc * kTcK ? a.ecol[k] : 0;
    if (warp == 0) {  // all 512 TMEM columns: 8 groups x 64 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    uint32_t ph_mma = 0, ph_cp = 0;
    bool failed = false;

    for (int tile = blockIdx.x; tile < a.n_tiles && !failed; tile += gridDim.x) {
        const int rt = tile / a.n_ct, ct = tile - rt * a.n_ct;
        const int row0 = rt * kTcRows;
        // 1. row exponents E_r (|b'_rk| < 2^(E_r - 1)) and non-finite rows; warp w takes rows w, w + 8, ...
        for (int rr = warp; rr < kTcRows; rr += kTcThreads / 32) {
            const int r = row0 + rr;
            int mx = -(1 << 29), bad = 0;
            if (r < a.n) {
                for (int k = lane; k < a.m; k += 32) {
                    const double x = a.B[(size_t)r * a.ldb + k];
                    bad |= !isfinite(x);
                    mx = max(mx, exponent_of(x) + s_ek[k]);
                }
            }
            mx = __reduce_max_sync(0xffffffffu, mx);
            bad = __reduce_or_sync(0xffffffffu, bad);
            if (lane == 0) {
                s_erow[rr] = mx > -(1 << 28) ? mx + 2 : 0;
                s_bad[rr] = bad;
            }
        }
        if (tid < kTcCols) s_scale[tid] = a.cscale[ct * kTcCols + tid];
        __syncthreads();
        for (int kc = 0; kc < a.n_kc; ++kc) {
            // 2. column digits of this (column tile, K chunk): 8 planes, 64 KB, by the bulk-copy engine
            if (tid == 0) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_cp),
                             "r"(kDigits * kPlaneB)
                             : "memory");
                const unsigned char* src =
                    reinterpret_cast<const unsigned char*>(a.digits) + (size_t)(ct * a.n_kc + kc) * kDigits * kPlaneB;
                for (int t = 0; t < kDigits; ++t)
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            sB + t * kPlaneB),
                        "l"(src + (size_t)t * kPlaneB), "r"(kPlaneB), "r"(bar_cp)
                        : "memory");
            }
            // 3. row digits: thread item = (row, 8 consecutive k), 8 planes of 16-byte stores
            for (int item = tid; item < kTcRows * (kTcK / 8); item += kTcThreads) {
                const int rr = item >> 3, kg = item & 7;
                const int r = row0 + rr, k0 = kc * kTcK + kg * 8;
                const int E = s_erow[rr];
                uint32_t w[kDigits][4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    int q0[kDigits], q1[kDigits];
                    const int ka = k0 + e, kb = k0 + e + 1;
                    const double xa = (r < a.n && ka < a.m) ? a.B[(size_t)r * a.ldb + ka] : 0.0;
                    const double xb = (r < a.n && kb < a.m) ? a.B[(size_t)r * a.ldb + kb] : 0.0;
                    base128_digits(fixed_point(xa, 56 - E + s_ek[ka]), q0);
                    base128_digits(fixed_point(xb, 56 - E + s_ek[kb]), q1);
#pragma unroll
                    for (int s = 0; s < kDigits; ++s) w[s][e >> 1] = bf16_bits(q0[s]) | (bf16_bits(q1[s]) << 16);
                }
                const int off = plane_off(rr, kg * 8);
#pragma unroll
                for (int s = 0; s < kDigits; ++s)
                    *reinterpret_cast<uint4*>(sm + kSmA + s * kPlaneA + off) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            __syncthreads();
            // 4. one thread issues the MMAs: every digit pair (s, t) with s + t <= 9 into group s + t
            if (tid == 0) {
                tc_fence_after();
                if (!mbar_wait(bar_cp, ph_cp)) {
                    atomicOr(a.err, kErrTimeout);
                    *s_flag = 1;
                    mbar_wait(bar_cp, ph_cp);  // one more bounded wait for the copies in flight
                } else {
#pragma unroll 1
                    for (int s = 0; s < kDigits; ++s) {
#pragma unroll 1
                        for (int t = 0; s + t < kGroups; ++t) {
                            const int g = s + t;
                            const uint32_t d = tmem + (uint32_t)(g * kTcCols);
#pragma unroll
                            for (int ks = 0; ks < kTcK / 16; ++ks) {
                                // the first product into a group overwrites it (new tile), later ones add
                                const uint32_t acc = (kc > 0 || ks > 0 || s > 0) ? 1u : 0u;
                                mma_bf16(d, smem_desc(sA + s * kPlaneA + ks * 256), smem_desc(sB + t * kPlaneB + ks * 256),
                                         acc);
                            }
                        }
                    }
                    mma_commit(bar_mma);
                }
            }
            ph_cp ^= 1u;
            __syncthreads();
            if (*s_flag) {
                failed = true;
                break;
            }
            // 5. the MMAs have read the digit planes (and written TMEM) before anything is overwritten
            const bool ok = mbar_wait(bar_mma, ph_mma);
            ph_mma ^= 1u;
            if (!ok) *s_flag = 1;
            __syncthreads();
            if (*s_flag) {
                if (tid == 0) atomicOr(a.err, kErrTimeout);
                failed = true;
                break;
            }
        }
        if (failed) break;
        // 6. epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows), columns 32 (w / 4) .. + 31
        tc_fence_after();
        {
            const int quarter = warp & 3, half = warp >> 2;
            const int rr = quarter * 32 + lane;
            const int r = row0 + rr;
            float best = 0.f;
#pragma unroll 1
            for (int c16 = 0; c16 < 2; ++c16) {
                const int col0 = half * 32 + c16 * 16;
                uint32_t v[kGroups][16];
#pragma unroll
                for (int g = 0; g < kGroups; ++g)
                    tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * kTcCols + col0), v[g]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    long long A[kGroups];
#pragma unroll
                    for (int g = 0; g < kGroups; ++g) A[g] = (long long)__float2int_rn(__uint_as_float(v[g][j]));
                    // sum_g A_g 128^(7 - g') = H 2^28 + L, exactly (g' = 0 .. 7 for g = 2 .. 9)
                    long long H = ((A[0] * 128 + A[1]) * 128 + A[2]) * 128 + A[3];
                    long long L = ((A[4] * 128 + A[5]) * 128 + A[6]) * 128 + A[7];
                    const long long Lh = L >> 28;
                    const long long Ll = L - (Lh << 28);  // [0, 2^28)
                    H += Lh;
                    float mag;
                    if (H > -(1ll << 34) && H < (1ll << 34))
                        mag = fabsf(__ll2float_rn((H << 28) + Ll));
                    else
                        mag = fabsf(__fmaf_rn(__ll2float_rn(H), 268435456.0f, __ll2float_rn(Ll)));
                    best = fmaxf(best, mag * s_scale[col0 + j]);
                }
            }
            if (r < a.n) {
                double gam = scalbn((double)best, s_erow[rr]);
                if (s_bad[rr]) gam = (double)INFINITY;
                if (gam > 0.0) atomicMax(&a.gbits[r], (unsigned long long)__double_as_longlong(gam));
            }
        }
        // TMEM reads are complete before the next tile's MMAs overwrite it
        tc_fence_before();
        __syncthreads();
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

}  // namespace

size_t grade_tc_digit_bytes(int m) {
    const int n_ct = (m + kTcCols - 1) / kTcCols, n_kc = (m + kTcK - 1) / kTcK;
    return (size_t)n_ct * n_kc * kDigits * kPlaneB;
}

int launch_grade_tc_prep(int m, const double* A, const double* Ai, void* digits, int* ecol, float* cscale,
                         cudaStream_t st) {
    if (m < 1 || m > kMaxM) return -1;
    const int n_ct = (m + kTcCols - 1) / kTcCols, n_kc = (m + kTcK - 1) / kTcK;
    k_grade_tc_prep<<<1, 512, 0, st>>>(m, A, Ai, static_cast<uint16_t*>(digits), ecol, cscale, n_ct, n_kc);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_grade_tc(int n, int m, const double* B, int ldb, const void* digits, const int* ecol, const float* cscale,
                    unsigned long long* gbits, int* err, cudaStream_t st, int n_sm) {
    if (n <= 0) return 0;
    if (m < 1 || m > kMaxM) return -1;
    cudaMemsetAsync(gbits, 0, sizeof(unsigned long long) * (size_t)n, st);
    TcArgs a;
    a.n = n;
    a.m = m;
    a.ldb = ldb;
    a.n_ct = (m + kTcCols - 1) / kTcCols;
    a.n_kc = (m + kTcK - 1) / kTcK;
    a.n_tiles = ((n + kTcRows - 1) / kTcRows) * a.n_ct;
    a.B = B;
    a.digits = static_cast<const uint16_t*>(digits);
    a.ecol = ecol;
    a.cscale = cscale;
    a.gbits = gbits;
    a.err = err;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_grade_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmAlloc);
        attr = true;
    }
    const int grid = a.n_tiles < n_sm ? a.n_tiles : n_sm;
    k_grade_tc<<<grid, kTcThreads, kSmAlloc, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 2 : -1;
}

}  // namespace mtp
