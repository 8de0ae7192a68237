// Generated by paper_2007_08555_gb300/codegen.py for lev_max = 4. Do not edit.
#pragma once
#include "mtp_gen_common.h"
namespace mtpgen_L4 {
constexpr int L = 4, C = 1, V = 2, M = 2, NMU = 1, NUMAX = 0;
constexpr int NS32 = 1, NS64 = 1;
constexpr int FWD_ROWS = 1, ADJ_ROWS = 2;
constexpr int FWD_LAYERS = 1, ADJ_LAYERS = 1;
constexpr int PROGRAM_OPS = 1;
constexpr int FLOP_PAIR_MOMENTS = 2, FLOP_PAIR_ADJOINT = 4, FLOP_ATOM_PROGRAM = 6;
static const int level_table[] = {2,2,1,1,0,0,4,2,1,0,0,1,0,0};
constexpr int LEVEL_TABLE_LEN = 14;
static const int basis_value[] = {0,1};
static const unsigned char comp_mu[] = {0};
static const unsigned char comp_abc[] = {0,0,0};
constexpr int NWEIGHTS = 2;
static const float weights[] = {0.0,1.0};
static const unsigned long long fwd_ops[] = {3096229038784512ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull};
static const unsigned long long adj_ops[] = {2533274790461440ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2814749767172096ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull};
static const int fwd_layer_rows[] = {1};
static const int adj_layer_rows[] = {2};
static const int s32_begin[] = {0};
static const int s32_size[] = {1};
static const int s64_begin[] = {0};
static const int s64_size[] = {1};
#define MTPGEN_HAS_UNROLLED 1
template <bool WANT_B>
__device__ __forceinline__ float contract_unrolled(const float* __restrict__ src, float* __restrict__ dst, const float* __restrict__ xi, double* __restrict__ bout) {
  const float v0 = src[0];
  const float v1 = v0 * v0;
  float e = 0.f;
  e += xi[0] * v0;
  if (WANT_B) bout[0] = (double)v0;
  e += xi[1] * v1;
  if (WANT_B) bout[1] = (double)v1;
  float a1 = xi[1];
  float a0 = xi[0];
  a0 += v0 * a1;
  a0 += v0 * a1;
  dst[0] = a0;
  return e;
}
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
}  // namespace mtpgen_L4
