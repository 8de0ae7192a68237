// Neighbourhoods of Sec. 2.1 (Eq. 1): for every atom i all (j, s) with |x_j + s H - x_i| < R_cut.
//
// Cell lists per configuration: atoms are binned by fractional coordinate into n_k bins along
// each lattice direction (bin width >= R_cut unless the cell is thinner), and each atom visits
// the bins within c_k = ceil(R_cut / bin width) along every direction, periodic images included
// (small cells are visited several times with different image shifts).  Distances are first
// taken in float from bin-local coordinates as a prefilter; pairs within 1e-3 Angstrom of the
// cutoff are decided in double precision with the fixed operation order documented in mtp.h, so
// the lists are identical to a brute-force double-precision search.  The cell lists of a batch are
// built by one cooperative launch (phases separated by bounded grid barriers).  One block of the
// list kernel handles one bin at a time: the atoms of the surrounding bins are staged once in
// shared memory and every warp tests them for one atom of the bin, compacting the accepted pairs
// with a ballot.  The accepted keys are rank-sorted by (j, s); in the same pass each lane forms r_ij
// of its keys, exactly in double precision for the double path and in double-float arithmetic
// (error-free float transformations, ~2^-44 relative) rounded once to float for the float path, and
// writes the pair record (r_ij and j | species << 24) in slot-major layout.  Double-precision
// instructions are few and never divergent: on this part a warp-wide double-precision instruction
// costs many times a float one.  A last kernel records, for every pair, the slot of the reverse
// pair in the neighbour's list (used by the deterministic force gather).
#include <algorithm>
#include "mtp_internal.h"
#include "mtp_common.cuh"

namespace mtp {

namespace {

constexpr int kScanItems = 4;
constexpr int kScanThreads = 512;
constexpr int kScanBlock = kScanItems * kScanThreads;
constexpr int kMaxImageReach = 16;
constexpr int kMaxShift = 50;  // |wrap| per atom; image shifts then stay within +-117
constexpr double kBand = 1e-3;

__device__ __forceinline__ int find_cfg(const int* cfg_off, int K, int i) {
    int lo = 0, hi = K;  // cfg_off[lo] <= i < cfg_off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cfg_off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// Per-configuration geometry: inverse cell, perpendicular widths, bin counts and reach.
__device__ void cell_desc(int k, const double* cells, const int* cfg_off, double rsearch, CellDesc* d, int* bin_total,
                          int* err) {
    CellDesc D;
    const double* H = cells + 9 * (size_t)k;
    bool finite = true;
    for (int q = 0; q < 9; ++q) {
        D.H[q] = H[q];
        finite = finite && isfinite(H[q]);
    }
    // input checks: every geometry below stays finite-indexed for any input (a NaN converts to a
    // zero bin count, clamped to one bin), so bad cells are only reported here
    if (!finite) atomicOr(err, kErrNonFinite);
    // The degenerate-cell check in double; the inverse cell and the bin geometry in float: fractional
    // coordinates only place atoms in bins and lattice wraps, where the 1e-3 Angstrom band of the
    // search covers the float error, and every neighbour decision is taken in double elsewhere (a
    // double-precision division or square root costs many float operations on this part).
    {
        const double a = H[0], b = H[1], c = H[2], e = H[3], f = H[4], g = H[5], h = H[6], ii = H[7], jj = H[8];
        const double det = a * (f * jj - g * ii) - b * (e * jj - g * h) + c * (e * ii - f * h);
        // flat or degenerate cell: |det| <= 1e-9 |a_0| |a_1| |a_2|, compared squared (no square roots)
        const double q0 = a * a + b * b + c * c, q1 = e * e + f * f + g * g, q2 = h * h + ii * ii + jj * jj;
        if (finite && !(det * det > 1e-18 * q0 * q1 * q2)) atomicOr(err, kErrCell);
    }
    const float a = (float)H[0], b = (float)H[1], c = (float)H[2], e = (float)H[3], f = (float)H[4],
                g = (float)H[5], h = (float)H[6], ii = (float)H[7], jj = (float)H[8];
    const float det = a * (f * jj - g * ii) - b * (e * jj - g * h) + c * (e * ii - f * h);
    const float vol = fabsf(det);
    {
        const float id = 1.f / det;
        D.Hi[0] = (f * jj - g * ii) * id; D.Hi[1] = (c * ii - b * jj) * id; D.Hi[2] = (b * g - c * f) * id;
        D.Hi[3] = (g * h - e * jj) * id; D.Hi[4] = (a * jj - c * h) * id; D.Hi[5] = (c * e - a * g) * id;
        D.Hi[6] = (e * ii - f * h) * id; D.Hi[7] = (b * h - a * ii) * id; D.Hi[8] = (a * f - b * e) * id;
    }
    const float irs = 1.f / (float)rsearch;
    const float Hf[9] = {a, b, c, e, f, g, h, ii, jj};
    float w[3];
    for (int q = 0; q < 3; ++q) {
        const float* u = Hf + ((q + 1) % 3) * 3;
        const float* v = Hf + ((q + 2) % 3) * 3;
        const float cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
        w[q] = vol * rsqrtf(cx * cx + cy * cy + cz * cz);
        int nq = (int)floorf(w[q] * irs * (1.f - 1e-5f));  // bins no thinner than the search radius
        D.n[q] = nq < 1 ? 1 : (nq > 1024 ? 1024 : nq);
    }
    const long natoms = cfg_off[k + 1] - cfg_off[k];
    const long limit = natoms > 1 ? natoms : 1;
    while ((long)D.n[0] * D.n[1] * D.n[2] > limit) {  // never more bins than atoms
        int q = 0;
        if (D.n[1] > D.n[q]) q = 1;
        if (D.n[2] > D.n[q]) q = 2;
        D.n[q] = D.n[q] / 2 > 0 ? D.n[q] / 2 : 1;
        if (D.n[0] * D.n[1] * D.n[2] == 1) break;
    }
    for (int q = 0; q < 3; ++q) {
        // bins to visit: ceil((rsearch + band) / width) with width = w / n, rounded up with a margin
        int cq = (int)ceilf(((float)rsearch + (float)kBand) * (float)D.n[q] / w[q] * (1.f + 1e-5f));
        if (cq < 1) cq = 1;
        if (cq > kMaxImageReach) {
            atomicOr(err, kErrCellThin);
            cq = kMaxImageReach;
        }
        D.c[q] = cq;
        const float inq = 1.f / (float)D.n[q];
        D.inv_n[q] = inq;
        for (int t = 0; t < 3; ++t) {
            D.hn[3 * q + t] = Hf[3 * q + t] * inq;
            D.hhi[3 * q + t] = Hf[3 * q + t];
            D.hlo[3 * q + t] = (float)(H[3 * q + t] - (double)Hf[3 * q + t]);
        }
    }
    D.nbins = D.n[0] * D.n[1] * D.n[2];
    // each configuration's bins are one contiguous range; where it lies depends on the order of
    // the atomics, which changes nothing downstream (lists are sorted by (j, s))
    D.bin0 = atomicAdd(bin_total, D.nbins);
    d[k] = D;
}

// Bin of atom i: fractional coordinates from the inverse cell, the lattice wrap w (x - w H lies in
// the cell), its position relative to its bin's origin (float, for the prefilter) and the wrapped
// position as a float pair (for the double-float displacements).  Returns the global bin index.
__device__ int bin_atom(int i, int K, const double* pos, const int* types, int S, const int* cfg_off,
                        const CellDesc* d, int* cfg_of, int* atom_bin, int* atom_wrap, float4* local, float4* wp,
                        int* err) {
    const int k = find_cfg(cfg_off, K, i);
    cfg_of[i] = k;
    if (types[i] < 0 || types[i] >= S) atomicOr(err, kErrSpecies);
    const CellDesc& D = d[k];
    const double x[3] = {pos[3 * (size_t)i], pos[3 * (size_t)i + 1], pos[3 * (size_t)i + 2]};
    // a non-finite position is reported; its bin and wrap below are clamped, and its pairs fail
    // every distance test, so no index is derived from it
    if (!(isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]))) atomicOr(err, kErrNonFinite);
    // bin and lattice wrap from float fractional coordinates (a bin slightly off is covered by the
    // band); the wrapped position x - w H in double, kept as a float pair (hi, lo) for the
    // double-float displacements, and the position relative to the bin's origin in float
    int w[3], b[3];
    const float xf[3] = {(float)x[0], (float)x[1], (float)x[2]};
    for (int q = 0; q < 3; ++q) {
        const float fq = xf[0] * D.Hi[0 * 3 + q] + xf[1] * D.Hi[1 * 3 + q] + xf[2] * D.Hi[2 * 3 + q];
        const float fl = floorf(fq);
        w[q] = (int)fl;
        const float fr = fq - fl;
        int bq = (int)(fr * (float)D.n[q]);
        if (bq < 0) bq = 0;
        if (bq >= D.n[q]) bq = D.n[q] - 1;
        b[q] = bq;
        if (w[q] > kMaxShift || w[q] < -kMaxShift) atomicOr(err, kErrShift);
    }
    double xw[3] = {x[0], x[1], x[2]};
    if (w[0] | w[1] | w[2])
        for (int t = 0; t < 3; ++t) xw[t] -= w[0] * D.H[0 * 3 + t] + w[1] * D.H[1 * 3 + t] + w[2] * D.H[2 * 3 + t];
    float hi[3], lo[3], lc[3];
    for (int t = 0; t < 3; ++t) {
        hi[t] = (float)xw[t];
        lo[t] = (float)(xw[t] - (double)hi[t]);
        const float o = (float)b[0] * D.hn[0 * 3 + t] + (float)b[1] * D.hn[1 * 3 + t] + (float)b[2] * D.hn[2 * 3 + t];
        lc[t] = (hi[t] - o) + lo[t];
    }
    local[i] = make_float4(lc[0], lc[1], lc[2], 0.f);
    wp[2 * (size_t)i] = make_float4(hi[0], hi[1], hi[2], 0.f);
    wp[2 * (size_t)i + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
    const int bin = D.bin0 + (b[0] * D.n[1] + b[1]) * D.n[2] + b[2];
    atom_bin[i] = bin;
    atom_wrap[i] = ((w[0] + 128) & 255) | (((w[1] + 128) & 255) << 8) | (((w[2] + 128) & 255) << 16);
    return bin;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Barrier over the whole grid of a cooperative launch (every block resident).  Barrier number
// `phase` (1, 2, ...) completes when the counter, zero at launch, reaches phase x gridDim.x.  The
// wait gives up after ~1 s: it sets kErrTimeout and returns false, and the block then leaves the
// kernel (the blocks still waiting give up the same way).
__device__ bool grid_barrier(int* ctr, int phase, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1);
        const int target = phase * (int)gridDim.x;
        const unsigned long long t0 = now_ns();
        int ok = 1;
        while (ld_acquire(ctr) < target) {
            if (now_ns() - t0 > 1000000000ull) {
                atomicOr(err, kErrTimeout);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

struct BinArgs {
    int K, n, S, n_zero;
    double rsearch;
    const double* cells;
    const int* cfg_off;
    const double* pos;
    const int* types;
    CellDesc* desc;
    int* counters;  // [0] bins handed out, [1] atoms handed out, [6] grid barrier (zero at launch)
    int* cfg_of;
    int* atom_bin;
    int* atom_wrap;
    int* atom_slot;
    float4* local;
    float4* wp;
    int* bin_count;
    int* bin_start;
    int* bin_atoms;
    int* err;
};

constexpr int kBinThreads = 128;

// The cell lists of a batch in one cooperative launch, four phases separated by grid barriers:
//   0. per configuration: geometry and its range of bins; every bin counter cleared;
//   1. per atom: its bin and wrap, and its slot in the bin (an atomic on the bin's counter);
//   2. per bin: its start in bin_atoms (a warp-wide scan, one atomic per warp on the running total;
//      the placement order changes nothing downstream);
//   3. per atom: bin_atoms[start of its bin + its slot] = i.
__global__ void __launch_bounds__(kBinThreads) k_bin_all(const BinArgs a) {
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    int* ctr = a.counters + 6;
    for (int k = t0; k < a.K; k += stride) cell_desc(k, a.cells, a.cfg_off, a.rsearch, a.desc, a.counters, a.err);
    for (int t = t0; t < a.n_zero; t += stride) a.bin_count[t] = 0;
    if (!grid_barrier(ctr, 1, a.err)) return;
    for (int i = t0; i < a.n; i += stride) {
        const int bin = bin_atom(i, a.K, a.pos, a.types, a.S, a.cfg_off, a.desc, a.cfg_of, a.atom_bin, a.atom_wrap,
                                 a.local, a.wp, a.err);
        a.atom_slot[i] = atomicAdd(&a.bin_count[bin], 1);
    }
    if (!grid_barrier(ctr, 2, a.err)) return;
    {
        const int nbins = ld_acquire(a.counters);  // bins handed out in phase 0
        const int lane = threadIdx.x & 31;
        for (int b0 = t0 & ~31; b0 < nbins; b0 += stride) {
            const int b = b0 + lane;
            const int c = b < nbins ? a.bin_count[b] : 0;
            int incl = c;
#pragma unroll
            for (int sh = 1; sh < 32; sh <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, sh);
                if (lane >= sh) incl += y;
            }
            int base = 0;
            if (lane == 31) base = atomicAdd(a.counters + 1, incl);
            base = __shfl_sync(0xffffffffu, base, 31);
            if (b < nbins) a.bin_start[b] = base + incl - c;
        }
    }
    if (!grid_barrier(ctr, 3, a.err)) return;
    pdl_trigger();  // the neighbour-list kernel may start launching
    for (int i = t0; i < a.n; i += stride) a.bin_atoms[a.bin_start[a.atom_bin[i]] + a.atom_slot[i]] = i;
}

__device__ __forceinline__ int unpack(int packed, int q) { return ((packed >> (8 * q)) & 255) - 128; }

// exact decision and displacement, written in the documented double-precision order
__device__ __forceinline__ double exact_r2(const double* xi, const double* xj, const double* H, const int* s,
                                           double* d) {
    for (int k = 0; k < 3; ++k) {
        double sh = __dmul_rn((double)s[0], H[0 * 3 + k]);
        sh = __dadd_rn(sh, __dmul_rn((double)s[1], H[1 * 3 + k]));
        sh = __dadd_rn(sh, __dmul_rn((double)s[2], H[2 * 3 + k]));
        d[k] = __dsub_rn(__dadd_rn(xj[k], sh), xi[k]);
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

struct BuildArgs {
    int n, cap, S;
    const int* nbins;  // bins handed out by the binning (its counter; empty bins are skipped)
    double rs2;      // rsearch^2 (double)
    float lo2, hi2;  // (rsearch -/+ band)^2
    const double* pos;
    const int* types;
    const int* cfg_of;
    const CellDesc* desc;
    const int* atom_bin;
    const int* atom_wrap;
    const float4* local;
    const float4* wp;
    const int* bin_start;
    const int* bin_count;
    const int* bin_atoms;
    int* count;
    void* pr;                     // [cap][n] PairRec<T>: r_ij and j | species << 24, slot-major
    unsigned long long* keys_am;  // [n][cap] the sorted keys, atom-major
    int* err;
    int* max_seen;
    const int* bin_barrier;  // the cell lists are complete when it equals bin_barrier_done
    int bin_barrier_done;
};

// ---- double-float arithmetic (float pairs hi + lo), error-free transformations -------------------
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_scale(float t, float hhi, float hlo) {  // t small integer
    const float p = __fmul_rn(t, hhi);
    const float e = __fmaf_rn(t, hhi, -p);
    return fast_two_sum(p, __fmaf_rn(t, hlo, e));
}

__device__ __forceinline__ int pack3(int s0, int s1, int s2) {
    return ((s0 + 128) & 255) | (((s1 + 128) & 255) << 8) | (((s2 + 128) & 255) << 16);
}
// image shift inside a pair key: s_0 in the high byte, so that keys sort by (j, s_0, s_1, s_2)
__device__ __forceinline__ int key_shift(int s0, int s1, int s2) { return pack3(s2, s1, s0); }
__device__ __forceinline__ int key_s(int packed, int q) { return unpack(packed, 2 - q); }
constexpr int kBias3 = 0x808080;  // three zero components

// Shared-memory layout of k_build (bytes): staged candidates, the current group of neighbour bins,
// then per warp the accepted keys and the lattice shift of the neighbour's bin of each.
constexpr int kBuildThreads = 128, kBuildWarps = kBuildThreads / 32;
constexpr int kGroup = kBuildThreads;  // neighbour bins described per staging round
constexpr int kChunk = 512;            // candidates staged per round
constexpr size_t kSmCpos = 0;
constexpr size_t kSmCshift = kSmCpos + sizeof(float4) * kChunk;
constexpr size_t kSmCtb = kSmCshift + sizeof(int) * kChunk;
constexpr size_t kSmGpre = kSmCtb + sizeof(int) * kChunk;
constexpr size_t kSmGstart = kSmGpre + sizeof(int) * (kGroup + 4);
constexpr size_t kSmGtb = kSmGstart + sizeof(int) * kGroup;
constexpr size_t kSmGoff = kSmGtb + sizeof(int) * kGroup;
constexpr size_t kSmWsum = kSmGoff + sizeof(float) * 3 * kGroup;
constexpr size_t kSmWarp = kSmWsum + 64;
size_t build_smem(int cap) { return kSmWarp + (size_t)kBuildWarps * cap * (8 + 4); }

// One block per bin (grid-stride over the bins).  The atoms of the bins around it are the candidates
// of every atom in it: they are staged once in shared memory (positions relative to the bin's
// origin, image shift minus the candidate's wrap), then each warp takes one atom of the bin, tests
// the staged candidates with its lanes and compacts the accepted ones with a ballot.  Small cells
// whose candidates exceed one staging round are re-staged for every group of four atoms.
template <class T>
__global__ void __launch_bounds__(kBuildThreads) k_build(const BuildArgs a) {
    pdl_enter();
    if (*a.bin_barrier != a.bin_barrier_done) {  // the binning gave up (error word set): empty lists
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) a.count[i] = 0;
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* cpos = reinterpret_cast<float4*>(smem_raw + kSmCpos);
    int* cshift = reinterpret_cast<int*>(smem_raw + kSmCshift);
    int* ctb = reinterpret_cast<int*>(smem_raw + kSmCtb);
    int* gpre = reinterpret_cast<int*>(smem_raw + kSmGpre);
    int* gstart = reinterpret_cast<int*>(smem_raw + kSmGstart);
    int* gtb = reinterpret_cast<int*>(smem_raw + kSmGtb);
    float* goff = reinterpret_cast<float*>(smem_raw + kSmGoff);
    int* wsum = reinterpret_cast<int*>(smem_raw + kSmWsum);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem_raw + kSmWarp) + (size_t)warp * a.cap;
    // lattice shift t = s + w_j - w_i of each accepted pair (the shift of the neighbour's bin)
    int* ktb = reinterpret_cast<int*>(reinterpret_cast<unsigned long long*>(smem_raw + kSmWarp) +
                                      (size_t)kBuildWarps * a.cap) + (size_t)warp * a.cap;
    PairRec<T>* PR = static_cast<PairRec<T>*>(a.pr);
    const size_t n = (size_t)a.n;
    __shared__ int smax;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    const int nbins = *a.nbins;
    for (int bin = blockIdx.x; bin < nbins; bin += gridDim.x) {
        const int nat = a.bin_count[bin];
        if (nat == 0) continue;
        const int start = a.bin_start[bin];
        const int k = a.cfg_of[a.bin_atoms[start]];
        const CellDesc& D = a.desc[k];
        const int lb = bin - D.bin0;
        const int b2 = lb % D.n[2], b1 = (lb / D.n[2]) % D.n[1], b0 = lb / (D.n[2] * D.n[1]);
        const int ny = 2 * D.c[1] + 1, nz = 2 * D.c[2] + 1;
        const int n_off = (2 * D.c[0] + 1) * ny * nz;
        // the visited bins are distinct (no bin seen through two images): each j is a candidate once
        const bool uniq = D.n[0] > 2 * D.c[0] && D.n[1] > 2 * D.c[1] && D.n[2] > 2 * D.c[2];
        bool reuse = false;  // the previous group of atoms left every candidate staged
        int total = 0;
        for (int ab = 0; ab < nat; ab += kBuildWarps) {
            const bool has = ab + warp < nat;
            const int i = has ? a.bin_atoms[start + ab + warp] : 0;
            const float4 li = has ? a.local[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            const int wi = has ? a.atom_wrap[i] : pack3(0, 0, 0);
            // the image shift of a pair is the staged (bin shift - w_j) plus w_i: biased bytes add
            // without carries as long as every component stays within +-127
            const int wik = key_shift(unpack(wi, 0), unpack(wi, 1), unpack(wi, 2)) - kBias3;
            int cnt = 0;
            for (int g0 = 0; g0 < n_off; g0 += kGroup) {
                if (!reuse) {
                    // 1a. this group's neighbour bins, one per thread: start, count, image shift of
                    //     the wrap, offset of its origin; then a block-wide exclusive scan of the counts
                    const int o = g0 + threadIdx.x;
                    int bstart = 0, bcnt = 0, tb0 = 0, tb1 = 0, tb2 = 0;
                    float ox = 0.f, oy = 0.f, oz = 0.f;
                    if (o < n_off) {
                        const int o2 = o % nz - D.c[2], o1 = (o / nz) % ny - D.c[1], o0 = o / (nz * ny) - D.c[0];
                        int w0 = b0 + o0, w1 = b1 + o1, w2 = b2 + o2;
                        while (w0 < 0) { w0 += D.n[0]; --tb0; }
                        while (w0 >= D.n[0]) { w0 -= D.n[0]; ++tb0; }
                        while (w1 < 0) { w1 += D.n[1]; --tb1; }
                        while (w1 >= D.n[1]) { w1 -= D.n[1]; ++tb1; }
                        while (w2 < 0) { w2 += D.n[2]; --tb2; }
                        while (w2 >= D.n[2]) { w2 -= D.n[2]; ++tb2; }
                        ox = o0 * D.hn[0] + o1 * D.hn[3] + o2 * D.hn[6];
                        oy = o0 * D.hn[1] + o1 * D.hn[4] + o2 * D.hn[7];
                        oz = o0 * D.hn[2] + o1 * D.hn[5] + o2 * D.hn[8];
                        const int nbin = D.bin0 + (w0 * D.n[1] + w1) * D.n[2] + w2;
                        bstart = a.bin_start[nbin];
                        bcnt = a.bin_count[nbin];
                    }
                    int incl = bcnt;
#pragma unroll
                    for (int sh = 1; sh < 32; sh <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, sh);
                        if (lane >= sh) incl += y;
                    }
                    if (lane == 31) wsum[warp] = incl;
                    __syncthreads();
                    int wpre = 0;
                    total = 0;
#pragma unroll
                    for (int w = 0; w < kBuildWarps; ++w) {
                        const int v = wsum[w];
                        wpre += w < warp ? v : 0;
                        total += v;
                    }
                    gpre[threadIdx.x] = wpre + incl - bcnt;
                    gstart[threadIdx.x] = bstart;
                    gtb[threadIdx.x] = pack3(tb0, tb1, tb2);
                    goff[threadIdx.x] = ox;
                    goff[kGroup + threadIdx.x] = oy;
                    goff[2 * kGroup + threadIdx.x] = oz;
                    __syncthreads();
                }
                for (int c0 = 0; c0 < total; c0 += kChunk) {
                    const int m = min(kChunk, total - c0);
                    if (!reuse) {
                        // 1b. stage candidates c0 .. c0 + m: bin g holds candidate f when
                        //     gpre[g] <= f < gpre[g + 1] (the last g with gpre[g] <= f)
                        for (int f = threadIdx.x; f < m; f += kBuildThreads) {
                            const int ff = c0 + f;
                            int g = 0;
#pragma unroll
                            for (int step = kGroup / 2; step > 0; step >>= 1)
                                if (gpre[g + step] <= ff) g += step;
                            const int j = a.bin_atoms[gstart[g] + (ff - gpre[g])];
                            const int wj = a.atom_wrap[j];
                            const float4 lj = a.local[j];
                            cpos[f] = make_float4(lj.x + goff[g], lj.y + goff[kGroup + g], lj.z + goff[2 * kGroup + g],
                                                  __int_as_float(j));
                            const int tb = gtb[g];
                            int tz = a.types[j];
                            tz = tz < 0 ? 0 : (tz >= a.S ? a.S - 1 : tz);  // invalid species are reported by the binning
                            // the key's low word: image shift in bytes 0..2, the neighbour's species in byte 3
                            // (a function of j: the key order stays (j, s))
                            cshift[f] = key_shift(unpack(tb, 0) - unpack(wj, 0), unpack(tb, 1) - unpack(wj, 1),
                                                  unpack(tb, 2) - unpack(wj, 2)) | (tz << 24);
                            ctb[f] = tb;
                        }
                        __syncthreads();
                    }
                    if (has) {
                        // 1c. float prefilter on the staged candidates, two per lane per round (their
                        //     shared-memory loads overlap); only the rare pairs within 1e-3 Angstrom of
                        //     the cutoff take the double-precision decision
                        auto test = [&](int e, bool& acc, unsigned long long& key, int& tbe) {
                            acc = false;
                            key = 0;
                            tbe = 0;
                            if (e >= m) return;
                            const float4 cp = cpos[e];
                            const float dx = cp.x - li.x, dy = cp.y - li.y, dz = cp.z - li.z;
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 > a.hi2) return;
                            const int j = __float_as_int(cp.w);
                            const int ks = cshift[e] + wik;  // key-order shift s (species in byte 3)
                            if (j == i && (ks & 0xffffff) == kBias3) return;
                            if (r2 < a.lo2) {
                                acc = true;
                            } else {
                                const int sv[3] = {key_s(ks, 0), key_s(ks, 1), key_s(ks, 2)};
                                const double xi[3] = {a.pos[3 * (size_t)i], a.pos[3 * (size_t)i + 1],
                                                      a.pos[3 * (size_t)i + 2]};
                                const double xj[3] = {a.pos[3 * (size_t)j], a.pos[3 * (size_t)j + 1],
                                                      a.pos[3 * (size_t)j + 2]};
                                double dd[3];
                                acc = exact_r2(xi, xj, D.H, sv, dd) < a.rs2;
                            }
                            key = ((unsigned long long)j << 32) | (unsigned long long)(unsigned)ks;
                            tbe = ctb[e];
                        };
                        for (int e0 = 0; e0 < m; e0 += 64) {
                            bool acc0, acc1;
                            unsigned long long key0, key1;
                            int tb0, tb1;
                            test(e0 + lane, acc0, key0, tb0);
                            test(e0 + 32 + lane, acc1, key1, tb1);
                            const unsigned b0 = __ballot_sync(0xffffffffu, acc0);
                            const unsigned b1 = __ballot_sync(0xffffffffu, acc1);
                            const unsigned below = (1u << lane) - 1u;
                            if (acc0) {
                                const int pos_ = cnt + __popc(b0 & below);
                                if (pos_ < a.cap) {
                                    keys[pos_] = key0;
                                    ktb[pos_] = tb0;
                                }
                            }
                            cnt += __popc(b0);
                            if (acc1) {
                                const int pos_ = cnt + __popc(b1 & below);
                                if (pos_ < a.cap) {
                                    keys[pos_] = key1;
                                    ktb[pos_] = tb1;
                                }
                            }
                            cnt += __popc(b1);
                        }
                    }
                    if (!reuse) __syncthreads();  // the next staging round overwrites the candidates
                }
            }
            reuse = n_off <= kGroup && total <= kChunk;
            if (!has) continue;
            __syncwarp();
            const int keep = min(cnt, a.cap);
            if (lane == 0) {
                if (cnt > a.cap) atomicOr(a.err, kErrOverflow);
                atomicMax(&smax, cnt);  // one global update per block, at the end
            }
            // 2. canonical order (j, s) by rank (keys are distinct), written in slot-major layout and
            //    atom-major for the reverse-pair search; each pass takes two keys per lane.  r_ij of
            //    each key: exact double precision for the double path, double-float arithmetic (then
            //    one rounding) for the float path; the neighbours' positions are loaded before the
            //    ranking, so their latency overlaps it.
            double xi[3] = {0.0, 0.0, 0.0};
            float4 pih = make_float4(0.f, 0.f, 0.f, 0.f), pil = pih;
            if (sizeof(T) == 8) {
                xi[0] = a.pos[3 * (size_t)i];
                xi[1] = a.pos[3 * (size_t)i + 1];
                xi[2] = a.pos[3 * (size_t)i + 2];
            } else {
                pih = a.wp[2 * (size_t)i];
                pil = a.wp[2 * (size_t)i + 1];
            }
            for (int e0 = 0; e0 < keep; e0 += 64) {
                const int ea = e0 + lane, eb = e0 + 32 + lane;
                const unsigned long long ka = ea < keep ? keys[ea] : ~0ull, kb = eb < keep ? keys[eb] : ~0ull;
                const int tba = ea < keep ? ktb[ea] : kBias3, tbb = eb < keep ? ktb[eb] : kBias3;
                // the neighbours' wrapped positions (float pairs) or positions (double)
                float4 jah = make_float4(0.f, 0.f, 0.f, 0.f), jal = jah, jbh = jah, jbl = jah;
                double xa[3] = {0.0, 0.0, 0.0}, xb[3] = {0.0, 0.0, 0.0};
                {
                    const size_t ja = ea < keep ? (size_t)(ka >> 32) : (size_t)i;
                    const size_t jb = eb < keep ? (size_t)(kb >> 32) : (size_t)i;
                    if (sizeof(T) == 8) {
                        for (int c = 0; c < 3; ++c) {
                            xa[c] = a.pos[3 * ja + c];
                            xb[c] = a.pos[3 * jb + c];
                        }
                    } else {
                        jah = a.wp[2 * ja];
                        jal = a.wp[2 * ja + 1];
                        jbh = a.wp[2 * jb];
                        jbl = a.wp[2 * jb + 1];
                    }
                }
                int ra = 0, rb = 0;
                if (uniq) {  // every j once: its index alone orders the keys (the high words)
                    const unsigned ja = (unsigned)(ka >> 32), jb = (unsigned)(kb >> 32);
                    const unsigned* kh = reinterpret_cast<const unsigned*>(keys) + 1;
#pragma unroll 4
                    for (int f = 0; f < keep; ++f) {
                        const unsigned jf = kh[2 * f];
                        ra += jf < ja ? 1 : 0;
                        rb += jf < jb ? 1 : 0;
                    }
                } else {
#pragma unroll 4
                    for (int f = 0; f < keep; ++f) {
                        const unsigned long long kf = keys[f];
                        ra += kf < ka ? 1 : 0;
                        rb += kf < kb ? 1 : 0;
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int e = h ? eb : ea;
                    if (e >= keep) continue;
                    const unsigned long long key = h ? kb : ka;
                    const int rank = h ? rb : ra;
                    const int j = (int)(key >> 32);
                    T r[3];
                    if (sizeof(T) == 8) {
                        const int sp = (int)(key & 0xffffffull);
                        const int sv[3] = {key_s(sp, 0), key_s(sp, 1), key_s(sp, 2)};
                        double dd[3];
                        exact_r2(xi, h ? xb : xa, D.H, sv, dd);
                        for (int c = 0; c < 3; ++c) r[c] = (T)dd[c];
                    } else {
                        // image shift relative to the wrapped positions, t = s + w_j - w_i: the lattice
                        // shift of the neighbour's bin, recorded when the pair was accepted
                        const int tb = h ? tbb : tba;
                        const float t[3] = {(float)unpack(tb, 0), (float)unpack(tb, 1), (float)unpack(tb, 2)};
                        const float4 pjh = h ? jbh : jah, pjl = h ? jbl : jal;
                        const float jh[3] = {pjh.x, pjh.y, pjh.z}, jl[3] = {pjl.x, pjl.y, pjl.z};
                        const float ih[3] = {pih.x, pih.y, pih.z}, il[3] = {pil.x, pil.y, pil.z};
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            DF d = df_add({jh[c], jl[c]}, {-ih[c], -il[c]});
#pragma unroll
                            for (int q = 0; q < 3; ++q)
                                if (t[q] != 0.f) d = df_add(d, df_scale(t[q], D.hhi[3 * q + c], D.hlo[3 * q + c]));
                            r[c] = (T)__fadd_rn(d.hi, d.lo);
                        }
                    }
                    const size_t o = (size_t)rank * n + i;
                    const int tj = (int)((key >> 24) & 255);  // the neighbour's species, from the key
                    PairRec<T> rec;
                    rec.x = r[0];
                    rec.y = r[1];
                    rec.z = r[2];
                    rec.jz = j | (tj << 24);
                    PR[o] = rec;  // one vector store per pair
                    a.keys_am[(size_t)i * a.cap + rank] = key;
                }
            }
            if (lane == 0) a.count[i] = keep;
            __syncwarp();
        }
        __syncthreads();  // the next bin stages over these candidates
    }
    if (threadIdx.x == 0 && smax > 0) atomicMax(a.max_seen, smax);
}

// one thread per (slot, atom): binary search of the reverse pair (i, -s) in the neighbour's sorted
// keys, stored atom-major so that one search stays within a few cache lines; rev starts at -1
__global__ void k_reverse(int n, int cap, int S, const int* types, const int* count, const int* jz, int jz_stride,
                          const unsigned long long* keys_am, int* rev) {
    const size_t N = (size_t)n;
    const size_t total = N * (size_t)cap;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < total; o += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(o / N);
        const int i = (int)(o - (size_t)p * N);
        if (p >= count[i]) continue;
        const int j = jz[o * jz_stride] & 0xffffff;
        const int sp = (int)(keys_am[(size_t)i * cap + p] & 0xffffffull);
        const int neg = ((256 - (sp & 255)) & 255) | (((256 - ((sp >> 8) & 255)) & 255) << 8) |
                        (((256 - ((sp >> 16) & 255)) & 255) << 16);
        // each pair is searched once, from its canonical side (i < j, or s above -s for an atom's
        // own images), which writes both slots; a pair without a partner keeps -1 (set before)
        if (!(i < j || (i == j && sp > neg))) continue;
        int zi = types[i];
        zi = zi < 0 ? 0 : (zi >= S ? S - 1 : zi);
        const unsigned long long want =
            ((unsigned long long)i << 32) | (unsigned long long)(unsigned)(neg | (zi << 24));
        const unsigned long long* kj = keys_am + (size_t)j * cap;
        int lo = 0, hi = count[j] - 1, found = -1;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            const unsigned long long key = kj[mid];
            if (key == want) {
                found = mid;
                break;
            }
            if (key < want) lo = mid + 1; else hi = mid - 1;
        }
        rev[o] = found;
        if (found >= 0) rev[(size_t)found * N + j] = p;
    }
}

// ---------------------------------------------------------------------------------------------
// exclusive scan
// ---------------------------------------------------------------------------------------------
__global__ void k_scan_blocks(const int* in, int* out, int n, int* block_sums) {
    __shared__ int warp_tot[kScanThreads / 32];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
    int v[kScanItems];
    int local = 0;
    for (int t = 0; t < kScanItems; ++t) {
        v[t] = (base + t < n) ? in[base + t] : 0;
        local += v[t];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int wt = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wt, o);
            if (lane >= o) wt += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = wt;
    }
    __syncthreads();
    int run = incl - local + (warp > 0 ? warp_tot[warp - 1] : 0);
    for (int t = 0; t < kScanItems; ++t) {
        if (base + t < n) out[base + t] = run;
        run += v[t];
    }
    if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = run;
}

__global__ void k_scan_sums(int* sums, int nb, int* total_out) {
    // one block: sequential over chunks of 1024
    __shared__ int carry;
    __shared__ int tmp[1024];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? sums[i] : 0;
        tmp[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int y = threadIdx.x >= o ? tmp[threadIdx.x - o] : 0;
            __syncthreads();
            tmp[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < nb) sums[i] = carry + tmp[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += tmp[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int* out, int n, const int* sums) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / kScanBlock];
}

__global__ void k_export(int n, int cap, const double* pos, const CellDesc* desc, const int* cfg_of, const int* count,
                         const int* jz, int jz_stride, const unsigned long long* keys_am, const int* offsets,
                         int* nbr_j, int* nbr_s,
                         double* r_ij) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const CellDesc& D = desc[cfg_of[i]];
    const double xi[3] = {pos[3 * (size_t)i], pos[3 * (size_t)i + 1], pos[3 * (size_t)i + 2]};
    const int cnt = count[i];
    for (int p = 0; p < cnt; ++p) {
        const size_t o = (size_t)p * n + i;
        const int j = jz[o * jz_stride] & 0xffffff;
        const int sp = (int)(keys_am[(size_t)i * cap + p] & 0xffffffull);  // slot p of the sorted keys
        const int s[3] = {((sp >> 16) & 255) - 128, ((sp >> 8) & 255) - 128, (sp & 255) - 128};
        const size_t q = (size_t)offsets[i] + p;
        nbr_j[q] = j;
        if (nbr_s)
            for (int t = 0; t < 3; ++t) nbr_s[3 * q + t] = s[t];
        if (r_ij) {
            const double xj[3] = {pos[3 * (size_t)j], pos[3 * (size_t)j + 1], pos[3 * (size_t)j + 2]};
            double d[3];
            exact_r2(xi, xj, D.H, s, d);
            for (int t = 0; t < 3; ++t) r_ij[3 * q + t] = d[t];
        }
    }
}

}  // namespace

// the jz words inside the pair records: a pointer to the first and the stride in ints
static const int* pair_jz(const NbrState& nb) {
    return nb.fp64 ? &nb.pr.as<PairRec<double>>()->jz : &nb.pr.as<PairRec<float>>()->jz;
}
static int jz_stride(const NbrState& nb) {
    return (int)((nb.fp64 ? sizeof(PairRec<double>) : sizeof(PairRec<float>)) / sizeof(int));
}

size_t scan_tmp_ints(int n) { return (size_t)(n + kScanBlock - 1) / kScanBlock + 8; }

int scan_exclusive(const int* in, int* out, int n, int* tmp, cudaStream_t st) {
    const int nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 0) {
        cudaMemsetAsync(out, 0, sizeof(int), st);
        return 1;
    }
    k_scan_blocks<<<nb, kScanThreads, 0, st>>>(in, out, n, tmp);
    k_scan_sums<<<1, 1024, 0, st>>>(tmp, nb, out + n);
    k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(out, n, tmp);
    return 3;
}

int build_neighbors(NbrState& nb, int K, int n, const int* cfg_off, const double* pos, const int* types,
                    const double* cells, double rsearch, bool fp64, int cap, cudaStream_t st, int S,
                    cudaStream_t side, cudaEvent_t fork, cudaEvent_t join) {
    int launches = 0;
    const size_t N = (size_t)n;
    const size_t bins_max = N + K + 1;
    const size_t recsz = fp64 ? sizeof(PairRec<double>) : sizeof(PairRec<float>);
    if (nb.count.reserve(N * 4) || nb.pr.reserve(N * cap * recsz) || nb.rev.reserve(N * cap * 4) ||
        nb.keys_am.reserve(N * cap * 8) || nb.cfg_of.reserve(N * 4) || nb.desc.reserve(sizeof(CellDesc) * K) ||
        nb.atom_bin.reserve(N * 4) || nb.atom_wrap.reserve(N * 4) || nb.atom_local.reserve(N * 16) || nb.atom_wp.reserve(N * 32) ||
        nb.bin_count.reserve(bins_max * 4) || nb.bin_start.reserve((bins_max + 1) * 4) ||
        nb.atom_slot.reserve(N * 4 + 4) || nb.bin_atoms.reserve(N * 4 + 4) ||
        nb.counters.reserve(64) ||
        nb.err.reserve(4))
        return -1;
    nb.n_atoms = n;
    nb.n_cfg = K;
    nb.cap = cap;
    nb.fp64 = fp64;
    nb.rsearch = rsearch;
    CellDesc* desc = nb.desc.as<CellDesc>();
    int* bin_count = nb.bin_count.as<int>();
    int* bin_start = nb.bin_start.as<int>();
    // counters: [0] bins handed out to configurations, [1] atoms handed out to bins, [2] largest
    // neighbour count seen, [4] and [5] the work queues of the moments and pair-gradient kernels
    int* counters = nb.counters.as<int>();
    cudaMemsetAsync(counters, 0, 8 * sizeof(int), st);
    const int total_bins_upper = n + K;  // every configuration has at most max(1, atoms) bins
    // the cell lists: one cooperative launch (its blocks wait on one another at grid barriers, so
    // all of them must be resident: the grid never exceeds the occupancy of the device)
    static int bin_occ = 0, n_sm = 0;
    if (!bin_occ) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bin_occ, k_bin_all, kBinThreads, 0);
        if (bin_occ < 1 || n_sm < 1) return -1;
    }
    const int bin_grid = std::max(1, std::min((std::max(n, K) + kBinThreads - 1) / kBinThreads, n_sm * bin_occ));
    {
        BinArgs b;
        b.K = K;
        b.n = n;
        b.S = S;
        b.n_zero = total_bins_upper + 1;
        b.rsearch = rsearch;
        b.cells = cells;
        b.cfg_off = cfg_off;
        b.pos = pos;
        b.types = types;
        b.desc = desc;
        b.counters = counters;
        b.cfg_of = nb.cfg_of.as<int>();
        b.atom_bin = nb.atom_bin.as<int>();
        b.atom_wrap = nb.atom_wrap.as<int>();
        b.atom_slot = nb.atom_slot.as<int>();
        b.local = nb.atom_local.as<float4>();
        b.wp = nb.atom_wp.as<float4>();
        b.bin_count = bin_count;
        b.bin_start = bin_start;
        b.bin_atoms = nb.bin_atoms.as<int>();
        b.err = nb.err.as<int>();
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)bin_grid);
        cfg.blockDim = dim3((unsigned)kBinThreads);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, k_bin_all, (const BinArgs)b) != cudaSuccess) return -1;
        ++launches;
    }
    BuildArgs a;
    a.n = n;
    a.cap = cap;
    a.S = S;
    a.rs2 = rsearch * rsearch;
    a.lo2 = (float)((rsearch - kBand) * (rsearch - kBand));
    a.hi2 = (float)((rsearch + kBand) * (rsearch + kBand));
    a.pos = pos;
    a.types = types;
    a.cfg_of = nb.cfg_of.as<int>();
    a.desc = desc;
    a.atom_bin = nb.atom_bin.as<int>();
    a.atom_wrap = nb.atom_wrap.as<int>();
    a.local = nb.atom_local.as<float4>();
    a.wp = nb.atom_wp.as<float4>();
    a.bin_start = bin_start;
    a.bin_count = bin_count;
    a.bin_atoms = nb.bin_atoms.as<int>();
    a.count = nb.count.as<int>();

    a.keys_am = nb.keys_am.as<unsigned long long>();
    a.pr = nb.pr.p;
    a.err = nb.err.as<int>();
    a.max_seen = nb.counters.as<int>() + 2;
    a.bin_barrier = nb.counters.as<int>() + 6;
    a.bin_barrier_done = 3 * bin_grid;
    a.nbins = counters;
    const size_t smem = build_smem(cap);
    // one block per bin when they fit in one wave (a perturbed lattice has ~12 atoms per bin)
    const int per_sm = (int)std::min<size_t>(12, (220 * 1024) / (smem + 1024));
    int blocks = std::min(total_bins_upper, 152 * std::max(per_sm, 1));
    if (blocks < 1) blocks = 1;
    const int threads = kBuildThreads;
    static int attr64 = 0, attr32 = 0;  // largest dynamic shared memory already allowed
    if (fp64) {
        if ((int)smem > attr64) {
            cudaFuncSetAttribute(k_build<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(k_build<double>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
            attr64 = (int)smem;
        }
        launch_pdl(k_build<double>, blocks, threads, smem, st, (const BuildArgs)a);
    } else {
        if ((int)smem > attr32) {
            cudaFuncSetAttribute(k_build<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(k_build<float>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
            attr32 = (int)smem;
        }
        launch_pdl(k_build<float>, blocks, threads, smem, st, (const BuildArgs)a);
    }
    ++launches;
    {
        const size_t total = N * (size_t)cap;
        size_t blocks = (total + 255) / 256;
        if (blocks > 152 * 64) blocks = 152 * 64;
        cudaStream_t rs = st;
        if (side) {  // overlaps the moments, contraction and pair-gradient kernels
            cudaEventRecord(fork, st);
            cudaStreamWaitEvent(side, fork, 0);
            rs = side;
        }
        cudaMemsetAsync(nb.rev.p, 0xff, sizeof(int) * total, rs);
        k_reverse<<<(int)blocks, 256, 0, rs>>>(n, cap, S, types, nb.count.as<int>(), pair_jz(nb), jz_stride(nb),
                                              nb.keys_am.as<unsigned long long>(), nb.rev.as<int>());
        if (side) cudaEventRecord(join, side);
    }
    ++launches;
    return cudaGetLastError() == cudaSuccess ? launches : -1;
}

int export_neighbors(const NbrState& nb, const double* pos, const int* offsets, int* nbr_j, int* nbr_s,
                     double* r_ij, cudaStream_t st) {
    const int n = nb.n_atoms;
    k_export<<<(n + 127) / 128, 128, 0, st>>>(n, nb.cap, pos, nb.desc.as<CellDesc>(), nb.cfg_of.as<int>(),
                                              nb.count.as<int>(), pair_jz(nb), jz_stride(nb),
                                              nb.keys_am.as<unsigned long long>(), offsets, nbr_j, nbr_s, r_ij);
    return 1;
}

}  // namespace mtp
