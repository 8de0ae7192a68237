// Generated by paper_2007_08555_gb300/codegen.py for lev_max = 2. Do not edit.
#pragma once
#include "mtp_gen_common.h"
namespace mtpgen_L2 {
constexpr int L = 2, C = 1, V = 1, M = 1, NMU = 1, NUMAX = 0;
constexpr int NS32 = 1, NS64 = 1;
constexpr int FWD_ROWS = 0, ADJ_ROWS = 0;
constexpr int FWD_LAYERS = 0, ADJ_LAYERS = 0;
constexpr int PROGRAM_OPS = 0;
constexpr int FLOP_PAIR_MOMENTS = 2, FLOP_PAIR_ADJOINT = 4, FLOP_ATOM_PROGRAM = 0;
static const int level_table[] = {1,2,1,1,0,0};
constexpr int LEVEL_TABLE_LEN = 6;
static const int basis_value[] = {0};
static const unsigned char comp_mu[] = {0};
static const unsigned char comp_abc[] = {0,0,0};
constexpr int NWEIGHTS = 0;
static const float weights[] = {};
static const unsigned long long fwd_ops[] = {0ull};
static const unsigned long long adj_ops[] = {0ull};
static const int fwd_layer_rows[] = {};
static const int adj_layer_rows[] = {};
static const int s32_begin[] = {0};
static const int s32_size[] = {1};
static const int s64_begin[] = {0};
static const int s64_size[] = {1};
#define MTPGEN_HAS_UNROLLED 0
template <int S> struct SliceF;
template <> struct SliceF<0> {
  static constexpr int BEGIN = 0, SIZE = 1;
  template <class T> static __device__ __forceinline__ void mom(const T x, const T y, const T z, const T* __restrict__ f, T* __restrict__ acc) {
    acc[0] += f[0] * T(1);
  }
  template <class T> static __device__ __forceinline__ void grad(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T* __restrict__ adj, T& s, T& gx, T& gy, T& gz) {
    { const T al = adj[0] * f[0]; const T be = adj[0] * df[0];
      s += be * T(1);
    }
  }
  template <class T> static __device__ __forceinline__ void tmom(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T rdu, const T ux, const T uy, const T uz, T* __restrict__ acc) {
    acc[0] += df[0] * rdu * T(1) + f[0] * (T(0));
  }
  template <class T> static __device__ __forceinline__ void pdot(const T x, const T y, const T z, const T* __restrict__ adjp, const T* __restrict__ adjtp, const T ux, const T uy, const T uz, T* __restrict__ P, T* __restrict__ Pd) {
    { const T av = adjp[0], atv = adjtp[0];
      P[0] += av * T(1); Pd[0] += atv * T(1) + av * (T(0)); }
  }
};
template <int S> struct SliceD;
template <> struct SliceD<0> {
  static constexpr int BEGIN = 0, SIZE = 1;
  template <class T> static __device__ __forceinline__ void mom(const T x, const T y, const T z, const T* __restrict__ f, T* __restrict__ acc) {
    acc[0] += f[0] * T(1);
  }
  template <class T> static __device__ __forceinline__ void grad(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T* __restrict__ adj, T& s, T& gx, T& gy, T& gz) {
    { const T al = adj[0] * f[0]; const T be = adj[0] * df[0];
      s += be * T(1);
    }
  }
  template <class T> static __device__ __forceinline__ void tmom(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T rdu, const T ux, const T uy, const T uz, T* __restrict__ acc) {
    acc[0] += df[0] * rdu * T(1) + f[0] * (T(0));
  }
  template <class T> static __device__ __forceinline__ void pdot(const T x, const T y, const T z, const T* __restrict__ adjp, const T* __restrict__ adjtp, const T ux, const T uy, const T uz, T* __restrict__ P, T* __restrict__ Pd) {
    { const T av = adjp[0], atv = adjtp[0];
      P[0] += av * T(1); Pd[0] += atv * T(1) + av * (T(0)); }
  }
};
struct Traits {
  static constexpr int L_ = L, C_ = C, V_ = V, M_ = M, NMU_ = NMU, NUMAX_ = NUMAX, NS32_ = NS32, NS64_ = NS64;
  template <int S> using F32 = SliceF<S>;
  template <int S> using F64 = SliceD<S>;
};
}  // namespace mtpgen_L2
