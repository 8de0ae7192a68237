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
//      written as 8 base-128 digits q_t (of b') and p_s (of G) (balanced, |digit| <= 65: exact in BF16);
//   3. for every digit pair (s, t) with s + t <= 7 the tensor cores form sum_k p_s,jk q_t,rk; pairs with
//      the same g = s + t share one FP32 accumulator (8 groups).  Each group sum is an integer below
//      8 x 460 x 65^2 < 2^24, so the FP32 accumulation is exact;
//   4. the epilogue combines the groups exactly in 64-bit integers,
//      sum_k T_r,k U_k,j = 2^49 sum_g A_g 128^(7-g) + (dropped pairs),
//      c_rj = 2^(E_r + F_j - 63) sum_g A_g 128^(7-g), rounds once to float and keeps the row maximum.
// Error: the rounding of b' and G to 56-bit grids and the dropped pairs (s + t >= 8) are each below
// ~1e-15 of 2^(E_r + F_j) (the scales of the row and the column), comparable to a double-precision
// product; the final rounding to float adds 2^-24 relative to gamma.  Rows holding NaN or inf get
// gamma = +inf.
//
// Shapes: the digits of G are the MMA's A operand (M = 128 output columns j per tile, so m <= 128
// takes one column tile), the digits of the rows of b its B operand (64 rows per tile).  The row
// digit planes of a K chunk sit in shared memory behind three zero planes, z_0..z_2 = 0 and
// z_(3+t) = q_t, each plane 64 rows x 32 k: for column digit s, the N = 256 window of planes
// 3 + 4h - s .. 6 + 4h - s holds q_(g-s) for the groups g = 4h .. 4h + 3, so one MMA accumulates the
// four pairs (s, g - s) into the TMEM columns of groups 4h .. 4h + 3 (TMEM lane = j, column
// = 64 g + r).  Per K step of 16 that is 12 MMAs of 128 x 256 (h = 0 only for s <= 3).
//
// Layout (shared memory, canonical K-major without swizzle): a plane of R rows x 32 k of BF16 is
// made of core matrices of 8 rows x 16 bytes; element (r, k) sits at
// (r / 8) * 512 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2 bytes (k groups 128 bytes apart: the
// descriptor's leading byte offset; row groups 512 bytes apart: its stride byte offset); planes of
// the same shape follow each other, so consecutive planes form one taller operand.
//
// One persistent CTA per SM (288 threads, ~227 KB of shared memory, all 512 TMEM columns) walks over
// row tiles of 64 and, for each, over the column tiles of 128; K is taken in chunks of 32 through two
// stages of shared memory.  Warp specialisation: one thread of the ninth warp copies the column
// digits of each chunk with the bulk-copy engine (cp.async.bulk, prepared once per active set),
// issues the chunk's 24 MMAs and commits them to the stage's mbarrier; the eight producer warps find
// the row exponents (for the next row tile while the tensor cores finish the current one), write the
// row digits of the next chunk into the other stage, and run the epilogue.  They meet only on
// mbarriers; every wait gives up after ~2 s and sets the error word, and the producers never branch
// on a wait's outcome, so every producer reaches every producer barrier.
#include <cuda_runtime.h>
#include <stdint.h>
#include "mtp_common.cuh"
#include "mtp_internal.h"

namespace mtp {

namespace {

constexpr int kTcThreads = 288;                // 8 producer / epilogue warps and one MMA warp
constexpr int kProd = 256;                     // producer threads
constexpr int kTcJ = 128;                      // M of the MMA: output columns j per tile
constexpr int kTcR = 64;                       // rows of b per tile (N = 4 x 64 per MMA)
constexpr int kTcK = 32;                       // K per chunk (two MMAs of K = 16)
constexpr int kStages = 2;                     // chunks in flight: digits of one while the other multiplies
constexpr int kDigits = 8;                     // base-128 digits per operand
constexpr int kGroups = 8;                     // g = s + t = 0 .. 7
constexpr int kZero = 3;                       // zero planes in front of the row digits
constexpr int kSbo = (kTcK / 8) * 128;         // bytes between 8-row groups of a plane
constexpr int kPlaneG = kTcJ * kTcK * 2;       // 8 KB: one digit plane of G (A operand)
constexpr int kPlaneQ = kTcR * kTcK * 2;       // 4 KB: one digit plane of the rows (B operand)
constexpr int kStageG = kDigits * kPlaneG;     // 64 KB
constexpr int kStageQ = (kZero + kDigits) * kPlaneQ;  // 44 KB
constexpr int kSmG = 0;
constexpr int kSmQ = kSmG + kStages * kStageG;
// barriers: [0,1] MMAs of a stage done, [2,3] its column digits landed, [4,5] its row digits written,
// [6] the epilogue has read TMEM
constexpr int kSmMisc = kSmQ + kStages * kStageQ;
constexpr int kMaxK = 512;                                 // K padded to whole chunks
constexpr int kMaxM = 480;  // exact FP32 group sums need 8 pairs x m x 65 x 64 < 2^24 (lev_max 20: m = 460)
constexpr int kSmEk = kSmMisc + 128;                       // int [kMaxK]
constexpr int kSmErow = kSmEk + 4 * kMaxK;                 // int [64]
constexpr int kSmBad = kSmErow + 4 * kTcR;                 // int [64]
constexpr int kSmScale = kSmBad + 4 * kTcR;                // float [128]
constexpr int kSmRed = kSmScale + 4 * kTcJ;                // [8][64] words: row-pass partials, row maxima
constexpr int kSmFlag = kSmRed + 4 * 8 * kTcR;             // int
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
    d |= (uint64_t)(((uint32_t)kSbo >> 4) & 0x3FFFu) << 32;  // stride byte offset: next 8 rows
    d |= (uint64_t)1 << 46;                           // descriptor version of this architecture
    return d;                                         // base offset 0, no swizzle
}

// instruction descriptor, kind::f16: D in F32, A and B in BF16, both K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((4 * kTcR) >> 3) << 17) |
                            ((uint32_t)(kTcJ >> 4) << 24);

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

// Byte offset of element (r, k) in a plane of kTcK columns (canonical K-major, no swizzle).
__host__ __device__ __forceinline__ int plane_off(int r, int k) {
    return (r >> 3) * kSbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
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

// NaN or infinity, from the exponent bits (integer work: no double-precision instruction)
__device__ __forceinline__ bool nonfinite(double x) {
    return (((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffu) == 0x7ffu;
}

// Eight base-128 digits of T (|T| < 2^55), most significant first: with U = T + 64 (1 + 128 + ...
// + 128^7), which makes every balanced digit non-negative, digit s of T is digit s of U minus 64
// (digits 2..8 in [-64, 63]); the first takes the rest of U (|q0| <= 65).  The two 28-bit halves
// of U give the digits with independent 32-bit shifts.
__device__ __forceinline__ void base128_digits(long long T, int* q) {
    constexpr long long kBias = 64ll * ((1ll << 56) - 1) / 127;  // 64 (1 + 128 + ... + 128^7)
    const long long U = T + kBias;
    const int lo = (int)(U & ((1ll << 28) - 1));
    const int hi = (int)(U >> 28);
#pragma unroll
    for (int s = 4; s < 8; ++s) q[s] = ((lo >> (7 * (7 - s))) & 127) - 64;
#pragma unroll
    for (int s = 1; s < 4; ++s) q[s] = ((hi >> (7 * (3 - s))) & 127) - 64;
    q[0] = (hi >> 21) - 64;
}

// A 64-bit unsigned integer rounded to the nearest float (ties to even), with integer operations
// only: the leading 24 bits after normalisation are the significand, the 40 bits below decide the
// rounding (a carry out of the significand moves into the exponent field by the addition).  The
// conversion instruction for 64-bit integers runs on the double-precision pipe of this part.
__device__ __forceinline__ float u64_to_float_rn(unsigned long long u) {
    if (u == 0ull) return 0.f;
    const int lz = __clzll((long long)u);
    const unsigned long long v = u << lz;  // bit 63 set
    unsigned int mant = (unsigned int)(v >> 40);
    const unsigned long long rem = v & ((1ull << 40) - 1ull);
    const unsigned long long half = 1ull << 39;
    mant += (rem > half || (rem == half && (mant & 1u))) ? 1u : 0u;
    const int e = 63 - lz;  // u in [2^e, 2^(e + 1))
    return __int_as_float(((e + 127) << 23) + (int)(mant - (1u << 23)));
}

// BF16 bits of a small integer (|d| < 2^8: exact)
__device__ __forceinline__ uint32_t bf16_bits(int d) {
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;  // exact for |d| < 2^22
    return __float_as_uint(f) >> 16;
}

// The digits of two elements as BF16 pairs: word s holds digit s of T0 (low half) and of T1 (high
// half).  The digit's bias is folded into the exponent trick: the float with the bits
// 0x4B400000 - 64 + u (u an unsigned base-128 digit of U, as in base128_digits) is 1.5 2^23 + u - 64,
// so subtracting 1.5 2^23 leaves the balanced digit exactly, and its BF16 is the upper half of its
// bits (one byte permutation packs two of them).
__device__ __forceinline__ void digit_pair_words(long long T0, long long T1, uint32_t* w) {
    constexpr long long kBias = 64ll * ((1ll << 56) - 1) / 127;
    const unsigned long long U0 = (unsigned long long)(T0 + kBias), U1 = (unsigned long long)(T1 + kBias);
    const unsigned lo0 = (unsigned)(U0 & ((1ull << 28) - 1)), lo1 = (unsigned)(U1 & ((1ull << 28) - 1));
    const unsigned hi0 = (unsigned)(U0 >> 28), hi1 = (unsigned)(U1 >> 28);
    auto bits = [](unsigned u) { return __float_as_uint(__uint_as_float(0x4B400000u - 64u + u) - 12582912.0f); };
#pragma unroll
    for (int s = 4; s < 8; ++s)
        w[s] = __byte_perm(bits((lo0 >> (7 * (7 - s))) & 127u), bits((lo1 >> (7 * (7 - s))) & 127u), 0x7632);
#pragma unroll
    for (int s = 1; s < 4; ++s)
        w[s] = __byte_perm(bits((hi0 >> (7 * (3 - s))) & 127u), bits((hi1 >> (7 * (3 - s))) & 127u), 0x7632);
    w[0] = __byte_perm(bits(hi0 >> 21), bits(hi1 >> 21), 0x7632);
}

// ------------------------------------------------------------------------------------------------
// Preparation once per active set: column exponents e_k of D, column scales F_j of G = (A D)^-1 and
// the digit planes of G in the layout of the MMA's A operand:
//   digits[((jt * n_kc + kc) * 8 + s) * 4096 + plane_off(j % 128, k % 32) / 2] = digit s of G_kj.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_grade_tc_prep(int m, const double* A, const double* Ai, uint16_t* digits,
                                                       int* ecol, float* cscale, int n_jt, int n_kc) {
    __shared__ int s_e[kMaxK];
    const int mpad = n_jt * kTcJ;
    // D_k = 2^e_k with max_r |A_rk| 2^e_k in [1/2, 1)
    for (int k = threadIdx.x; k < kMaxK; k += blockDim.x) {
        int e = 0;
        if (k < m) {
            int mx = -(1 << 29);
            for (int r = 0; r < m; ++r) mx = max(mx, exponent_of(A[(size_t)r * m + k]));
            e = mx > -(1 << 28) ? -(mx + 1) : 0;
        }
        s_e[k] = e;
        if (k < n_kc * kTcK) ecol[k] = e;
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
        const int jt = j / kTcJ, jj = j % kTcJ;
        for (int k = 0; k < n_kc * kTcK; ++k) {
            int q[kDigits] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (j < m && k < m) base128_digits(fixed_point(Ai[(size_t)k * m + j], 56 - F - s_e[k]), q);
            const int kc = k / kTcK, kk = k % kTcK;
            const size_t base = ((size_t)(jt * n_kc + kc) * kDigits) * (kPlaneG / 2) + plane_off(jj, kk) / 2;
#pragma unroll
            for (int t = 0; t < kDigits; ++t) digits[base + (size_t)t * (kPlaneG / 2)] = (uint16_t)bf16_bits(q[t]);
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

constexpr int kSmallSumsM = 127;

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kProd) : "memory"); }

// Nine warps share the four sub-partitions of an SM (three on one of them), which caps a thread at
// 168 registers.
__global__ void __launch_bounds__(kTcThreads, 1) k_grade_tc(const TcArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kSmMisc);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kSmMisc + 64);
    int* s_ek = reinterpret_cast<int*>(sm + kSmEk);
    int* s_erow = reinterpret_cast<int*>(sm + kSmErow);
    int* s_bad = reinterpret_cast<int*>(sm + kSmBad);
    float* s_scale = reinterpret_cast<float*>(sm + kSmScale);
    float* s_red = reinterpret_cast<float*>(sm + kSmRed);
    const uint32_t sG = smem_u32(sm + kSmG), sQ = smem_u32(sm + kSmQ);
    auto bar = [&](int q) { return smem_u32(&bars[q]); };

    if (tid == 0) {
        for (int q = 0; q < 2 * kStages; ++q) mbar_init(bar(q), 1);   // MMA commits, bulk copies
        for (int q = 0; q < kStages; ++q) mbar_init(bar(4 + q), kProd);  // row digits written
        mbar_init(bar(6), kProd);                                         // TMEM read by the epilogue
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int k = tid; k < kMaxK; k += kTcThreads) s_ek[k] = k < a.n_kc * kTcK ? a.ecol[k] : 0;
    // the zero planes in front of each stage's row digits (never written again)
    for (int st = 0; st < kStages; ++st)
        for (int e = tid; e < kZero * kPlaneQ / 16; e += kTcThreads)
            reinterpret_cast<uint4*>(sm + kSmQ + st * kStageQ)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) {  // all 512 TMEM columns: 8 groups x 64 rows
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zero planes, for the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int n_rt = (a.n + kTcR - 1) / kTcR;

    if (warp == kProd / 32) {
        // ---- MMA warp, one thread: bulk copies of the column digits and the MMAs, chunk by chunk ----
        if (lane == 0) {
            // phase parities and pending commits, one bit per stage (registers, not local memory)
            uint32_t ph_empty = 0u, ph_cp = 0u, ph_full = 0u, used = 0u, ph_tmem = 0u;
            bool ok = true, first_tile = true;
            for (int rt = blockIdx.x; rt < n_rt && ok; rt += gridDim.x) {
                for (int jt = 0; jt < a.n_ct && ok; ++jt) {
                    for (int kc = 0; kc < a.n_kc && ok; ++kc) {
                        const int st = kc & 1;
                        // the stage's previous MMAs have read its buffers
                        if ((used >> st) & 1u) {
                            ok = mbar_wait(bar(st), (ph_empty >> st) & 1u);
                            ph_empty ^= 1u << st;
                            used &= ~(1u << st);
                            if (!ok) break;
                        }
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(2 + st)),
                                     "r"(kStageG)
                                     : "memory");
                        const unsigned char* src =
                            reinterpret_cast<const unsigned char*>(a.digits) + (size_t)(jt * a.n_kc + kc) * kStageG;
                        for (int h = 0; h < 2; ++h)
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                    sG + st * kStageG + h * (kStageG / 2)),
                                "l"(src + (size_t)h * (kStageG / 2)), "r"(kStageG / 2), "r"(bar(2 + st))
                                : "memory");
                        // before the first MMA of a tile: the epilogue of the previous tile has read TMEM
                        if (kc == 0 && !first_tile) {
                            ok = mbar_wait(bar(6), ph_tmem);
                            ph_tmem ^= 1u;
                        }
                        first_tile = false;
                        // column digits landed and row digits written
                        ok = ok && mbar_wait(bar(2 + st), (ph_cp >> st) & 1u);
                        ph_cp ^= 1u << st;
                        ok = ok && mbar_wait(bar(4 + st), (ph_full >> st) & 1u);
                        ph_full ^= 1u << st;
                        if (!ok) break;
                        tc_fence_after();
                        // shared-memory addresses stay below 2^18, so offsets add to the descriptors'
                        // start-address field (addr >> 4, 14 bits) without carries
                        const uint64_t dg = smem_desc(sG + st * kStageG), dq = smem_desc(sQ + st * kStageQ);
#pragma unroll
                        for (int ks = 0; ks < kTcK / 16; ++ks) {
#pragma unroll
                            for (int sd = 0; sd < kDigits; ++sd) {
                                const uint32_t acc = (kc > 0 || ks > 0 || sd > 0) ? 1u : 0u;  // first overwrites
                                const uint64_t da = dg + (uint64_t)((sd * kPlaneG + ks * 256) >> 4);
#pragma unroll
                                for (int h = 0; h < 2; ++h) {
                                    if (h == 0 && sd > 3) continue;
                                    const int zs = kZero + 4 * h - sd;  // first plane of the window
                                    mma_bf16(tmem + (uint32_t)(h * 4 * kTcR), da,
                                             dq + (uint64_t)((zs * kPlaneQ + ks * 256) >> 4), acc);
                                }
                            }
                        }
                        mma_commit(bar(st));  // frees the stage; the tile's last commit releases the epilogue
                        used |= 1u << st;
                    }
                }
            }
            if (!ok) atomicOr(a.err, kErrTimeout);
            // leave no MMA or copy behind before the tensor memory is freed (bounded waits)
            for (int st = 0; st < kStages; ++st)
                if ((used >> st) & 1u) mbar_wait(bar(st), (ph_empty >> st) & 1u);
        }
        __syncwarp();
    } else {
        // ---- producers: row exponents, row digits, epilogue.  Their control flow never depends on a
        // wait's outcome, so every producer reaches every producer barrier; after a failed wait a
        // thread skips the remaining waits and the kernel's results are void (error word set). ----
        bool ok = true;
        uint32_t ph_done = 0u;  // phase parity of each stage's MMA barrier, one bit per stage
        // thread = (row rr of the tile, k group kg: 8 consecutive k of every chunk); the four threads of
        // a row are adjacent lanes
        const int rr = tid >> 2, kg = tid & 3;
        // Row exponents E_r (|b'_rk| < 2^(E_r - 1)) and non-finite rows of row tile t, combined over the
        // row's four threads by shuffles.  Called for the next row tile while the tensor cores finish
        // the current one.
        auto row_pass = [&](int t, int& E_out, int& bad_out) {
            const int r = t * kTcR + rr;
            const double* brow = a.B + (size_t)(r < a.n ? r : 0) * a.ldb;
            int mx = -(1 << 29), bad = 0;
            for (int c = 0; c < a.n_kc; c += 2) {
                double x[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int k = (c + (u >> 3)) * kTcK + kg * 8 + (u & 7);
                    x[u] = (r < a.n && k < a.m) ? brow[k] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int k = (c + (u >> 3)) * kTcK + kg * 8 + (u & 7);
                    if (k < a.m) {
                        bad |= nonfinite(x[u]);
                        mx = max(mx, exponent_of(x[u]) + s_ek[k]);
                    }
                }
            }
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
            bad |= __shfl_xor_sync(0xffffffffu, bad, 1);
            bad |= __shfl_xor_sync(0xffffffffu, bad, 2);
            E_out = mx > -(1 << 28) ? mx + 2 : 0;
            bad_out = bad;
        };
        int E = 0, bad_row = 0;
        if (blockIdx.x < n_rt) row_pass(blockIdx.x, E, bad_row);
        for (int rt = blockIdx.x; rt < n_rt; rt += gridDim.x) {
          const int row0 = rt * kTcR;
          const int r = row0 + rr;
          const double* brow = a.B + (size_t)(r < a.n ? r : 0) * a.ldb;
          if (kg == 0) {  // for the tile's final step (the previous one ended with a producer barrier)
              s_erow[rr] = E;
              s_bad[rr] = bad_row;
          }
          for (int jt = 0; jt < a.n_ct; ++jt) {
            if (tid < kTcJ) s_scale[tid] = a.cscale[jt * kTcJ + tid];
            producers_sync();  // row exponents and column scales visible to all producers
            for (int kc = 0; kc < a.n_kc; ++kc) {
                const int st = kc & 1;
                // 2. the stage is free once the MMAs that read it (two chunks back) are done
                if (kc >= 2) {
                    ok = ok && mbar_wait(bar(st), (ph_done >> st) & 1u);
                    ph_done ^= 1u << st;
                }
                // 3. row digits: thread = (row, 8 consecutive k), 8 planes of 16-byte stores behind the zeros
                {
                    unsigned char* Qs = sm + kSmQ + st * kStageQ + kZero * kPlaneQ;
                    const int k0 = kc * kTcK + kg * 8;
                    uint32_t w[kDigits][4];
                    double x[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) x[e] = (r < a.n && k0 + e < a.m) ? brow[k0 + e] : 0.0;
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        uint32_t pw[kDigits];
                        digit_pair_words(fixed_point(x[e], 56 - E + s_ek[k0 + e]),
                                         fixed_point(x[e + 1], 56 - E + s_ek[k0 + e + 1]), pw);
#pragma unroll
                        for (int q = 0; q < kDigits; ++q) w[q][e >> 1] = pw[q];
                    }
                    const int off = plane_off(rr, kg * 8);
#pragma unroll
                    for (int q = 0; q < kDigits; ++q)
                        *reinterpret_cast<uint4*>(Qs + q * kPlaneQ + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(bar(4 + st));  // this thread's digits of the chunk are written
            }
            // the next row tile's exponents, while the tensor cores finish this one
            if (jt == a.n_ct - 1 && rt + (int)gridDim.x < n_rt) row_pass(rt + gridDim.x, E, bad_row);
            // 4. the tile's MMAs are done: the commits of its last two chunks (one per stage)
            for (int kc = a.n_kc > 2 ? a.n_kc - 2 : 0; kc < a.n_kc; ++kc) {
                const int st = kc & 1;
                ok = ok && mbar_wait(bar(st), (ph_done >> st) & 1u);
                ph_done ^= 1u << st;
            }
            // 5. epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its columns j) and rows
            //    32 (w / 4) .. + 31 of the tile; the row maxima over j go through shared memory
            tc_fence_after();
            {
                const int quarter = warp & 3, halfr = warp >> 2;
                const int j = quarter * 32 + lane;
                // group sums stay below 2^22 for m <= 127: 8 pairs x m x 65 x 64 (digit bounds)
                const bool small_sums = a.m <= kSmallSumsM;
                const float scale = s_scale[j];
#pragma unroll 1
                for (int c16 = 0; c16 < 2; ++c16) {
                    const int r0 = halfr * 32 + c16 * 16;
                    uint32_t v[kGroups][16];
#pragma unroll
                    for (int g = 0; g < kGroups; ++g)
                        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * kTcR + r0), v[g]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (c16 == 1) {  // TMEM fully read: the next tile's MMAs may overwrite it
                        tc_fence_before();
                        mbar_arrive(bar(6));
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        // sum_g A_g 128^(7 - g) = H 2^28 + L, exactly, with H and L from the pairs
                        // X = A_0 128 + A_1, Y = A_2 128 + A_3 (and likewise for groups 4..7), which
                        // fit in 32 bits: |A_g| <= 8 m 65 64 = 15,974,400 for m = 480, so |X| <= 129
                        // times that, below 2^31
                        int A[kGroups];
                        if (small_sums) {
                            // A_g + 1.5 2^23 is exact in [2^23, 2^24) and its bits are 0x4B400000 + A_g
#pragma unroll
                            for (int g = 0; g < kGroups; ++g)
                                A[g] = (int)__float_as_uint(__uint_as_float(v[g][i]) + 12582912.0f) - 0x4B400000;
                        } else {
#pragma unroll
                            for (int g = 0; g < kGroups; ++g) A[g] = __float2int_rn(__uint_as_float(v[g][i]));
                        }
                        const long long H = ((long long)(A[0] * 128 + A[1]) << 14) + (A[2] * 128 + A[3]);
                        const long long L = ((long long)(A[4] * 128 + A[5]) << 14) + (A[6] * 128 + A[7]);
                        float mag;
                        if (H > -(1ll << 34) && H < (1ll << 34)) {  // |H 2^28 + L| < 2^63
                            const long long T = (H << 28) + L;
                            mag = u64_to_float_rn((unsigned long long)(T < 0 ? -T : T));
                        } else {
                            // beyond 64 bits: H' = H + floor(L / 2^28) and L' = L mod 2^28 in [0, 2^28);
                            // L' is below half an ulp of H' 2^28 (|H'| >= 2^33), so rounding H' is
                            // rounding the value (up to exact ties)
                            const long long Hn = H + (L >> 28);
                            const float hf = u64_to_float_rn((unsigned long long)(Hn < 0 ? -Hn : Hn));
                            mag = fabsf(__fmaf_rn(Hn < 0 ? -hf : hf, 268435456.0f, (float)(int)(L & ((1ll << 28) - 1))));
                        }
                        float v2 = mag * scale;
                        if (!(v2 >= 0.f)) v2 = 0.f;  // 0 x inf from a column scale beyond float range
                        // maximum over the warp's 32 columns j (non-negative floats order as their bits)
                        const unsigned mbits = __reduce_max_sync(0xffffffffu, __float_as_uint(v2));
                        if (lane == i) s_red[quarter * kTcR + r0 + i] = __uint_as_float(mbits);
                    }
                }
            }
            producers_sync();
            if (tid < kTcR) {
                const int r = row0 + tid;
                const float best = fmaxf(fmaxf(s_red[tid], s_red[kTcR + tid]), fmaxf(s_red[2 * kTcR + tid], s_red[3 * kTcR + tid]));
                if (r < a.n && ok) {
                    double gam = scalbn((double)best, s_erow[tid]);
                    if (s_bad[tid]) gam = (double)INFINITY;
                    if (gam > 0.0) atomicMax(&a.gbits[r], (unsigned long long)__double_as_longlong(gam));
                }
            }
            producers_sync();
          }
        }
        if (!ok) atomicOr(a.err, kErrTimeout);
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

}  // namespace

size_t grade_tc_digit_bytes(int m) {
    const int n_jt = (m + kTcJ - 1) / kTcJ, n_kc = (m + kTcK - 1) / kTcK;
    return (size_t)n_jt * n_kc * kStageG;
}

int launch_grade_tc_prep(int m, const double* A, const double* Ai, void* digits, int* ecol, float* cscale,
                         cudaStream_t st) {
    if (m < 1 || m > kMaxM) return -1;
    const int n_jt = (m + kTcJ - 1) / kTcJ, n_kc = (m + kTcK - 1) / kTcK;
    k_grade_tc_prep<<<1, 512, 0, st>>>(m, A, Ai, static_cast<uint16_t*>(digits), ecol, cscale, n_jt, n_kc);
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
    a.n_ct = (m + kTcJ - 1) / kTcJ;
    a.n_kc = (m + kTcK - 1) / kTcK;
    a.n_tiles = ((n + kTcR - 1) / kTcR) * a.n_ct;
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
    const int n_rt = (n + kTcR - 1) / kTcR;
    const int grid = n_rt < n_sm ? n_rt : n_sm;
    k_grade_tc<<<grid, kTcThreads, kSmAlloc, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 2 : -1;
}

}  // namespace mtp
