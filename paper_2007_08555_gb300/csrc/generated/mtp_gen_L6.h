// Generated by paper_2007_08555_gb300/codegen.py for lev_max = 6. Do not edit.
#pragma once
#include "mtp_gen_common.h"
namespace mtpgen_L6 {
constexpr int L = 6, C = 5, V = 8, M = 5, NMU = 2, NUMAX = 1;
constexpr int NS32 = 1, NS64 = 1;
constexpr int FWD_ROWS = 4, ADJ_ROWS = 5;
constexpr int FWD_LAYERS = 2, ADJ_LAYERS = 2;
constexpr int PROGRAM_OPS = 5;
constexpr int FLOP_PAIR_MOMENTS = 13, FLOP_PAIR_ADJOINT = 38, FLOP_ATOM_PROGRAM = 30;
static const int level_table[] = {5,2,1,1,0,0,4,2,1,0,0,1,0,0,6,1,1,1,0,6,1,2,0,1,0,1,1,6,3,1,0,0,1,0,0,1,0,0};
constexpr int LEVEL_TABLE_LEN = 38;
static const int basis_value[] = {0,6,1,5,7};
static const unsigned char comp_mu[] = {0,1,0,0,0};
static const unsigned char comp_abc[] = {0,0,0,0,0,0,1,0,0,0,1,0,0,0,1};
constexpr int NWEIGHTS = 2;
static const float weights[] = {0.0,1.0};
static const unsigned long long fwd_ops[] = {2533296265363458ull,3096250513620992ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2251821288718339ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2814771242205188ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,3096254808588294ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull};
static const unsigned long long adj_ops[] = {2533283380658178ull,2533287675625475ull,2533291970592772ull,3096250514079744ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2814758357368834ull,2814762652336131ull,2814766947303428ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2533274790789120ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2251799814078464ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2814749767565318ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull};
static const int fwd_layer_rows[] = {3,4};
static const int adj_layer_rows[] = {2,5};
static const int s32_begin[] = {0};
static const int s32_size[] = {5};
static const int s64_begin[] = {0};
static const int s64_size[] = {5};
#define MTPGEN_HAS_UNROLLED 1
template <bool WANT_B>
__device__ __forceinline__ float contract_unrolled(const float* __restrict__ src, float* __restrict__ dst, const float* __restrict__ xi, double* __restrict__ bout) {
  const float v0 = src[0];
  const float v1 = src[32];
  const float v2 = src[64];
  const float v3 = src[96];
  const float v4 = src[128];
  const float v5 = v2 * v2 + v3 * v3 + v4 * v4;
  const float v6 = v0 * v0;
  const float v7 = v6 * v0;
  float e = 0.f;
  e += xi[0] * v0;
  if (WANT_B) bout[0] = (double)v0;
  e += xi[1] * v6;
  if (WANT_B) bout[1] = (double)v6;
  e += xi[2] * v1;
  if (WANT_B) bout[2] = (double)v1;
  e += xi[3] * v5;
  if (WANT_B) bout[3] = (double)v5;
  e += xi[4] * v7;
  if (WANT_B) bout[4] = (double)v7;
  float a7 = xi[4];
  float a6 = xi[1];
  float a0 = xi[0];
  a6 += v0 * a7;
  a0 += v6 * a7;
  a0 += v0 * a6;
  a0 += v0 * a6;
  float a5 = xi[3];
  float a2 = 0.f;
  a2 += v2 * a5;
  a2 += v2 * a5;
  float a3 = 0.f;
  a3 += v3 * a5;
  a3 += v3 * a5;
  float a4 = 0.f;
  a4 += v4 * a5;
  a4 += v4 * a5;
  dst[0] = a0;
  float a1 = xi[2];
  dst[32] = a1;
  dst[64] = a2;
  dst[96] = a3;
  dst[128] = a4;
  return e;
}
template <int S> struct SliceF;
template <> struct SliceF<0> {
  static constexpr int BEGIN = 0, SIZE = 5;
  template <class T> static __device__ __forceinline__ void mom(const T x, const T y, const T z, const T* __restrict__ f, T* __restrict__ acc) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    acc[0] += f[0] * T(1);
    acc[1] += f[1] * T(1);
    acc[2] += f[0] * m1_0_0;
    acc[3] += f[0] * m0_1_0;
    acc[4] += f[0] * m0_0_1;
  }
  template <class T> static __device__ __forceinline__ void grad(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T* __restrict__ adj, T& s, T& gx, T& gy, T& gz) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    { const T al = adj[0] * f[0] + adj[1] * f[1]; const T be = adj[0] * df[0] + adj[1] * df[1];
      s += be * T(1);
    }
    { const T al = adj[2] * f[0]; const T be = adj[2] * df[0];
      s += be * m1_0_0;
      gx += al * T(1);
    }
    { const T al = adj[3] * f[0]; const T be = adj[3] * df[0];
      s += be * m0_1_0;
      gy += al * T(1);
    }
    { const T al = adj[4] * f[0]; const T be = adj[4] * df[0];
      s += be * m0_0_1;
      gz += al * T(1);
    }
  }
  template <class T> static __device__ __forceinline__ void tmom(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T rdu, const T ux, const T uy, const T uz, T* __restrict__ acc) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    acc[0] += df[0] * rdu * T(1) + f[0] * (T(0));
    acc[1] += df[1] * rdu * T(1) + f[1] * (T(0));
    acc[2] += df[0] * rdu * m1_0_0 + f[0] * (T(1) * ux);
    acc[3] += df[0] * rdu * m0_1_0 + f[0] * (T(1) * uy);
    acc[4] += df[0] * rdu * m0_0_1 + f[0] * (T(1) * uz);
  }
  template <class T> static __device__ __forceinline__ void pdot(const T x, const T y, const T z, const T* __restrict__ adjp, const T* __restrict__ adjtp, const T ux, const T uy, const T uz, T* __restrict__ P, T* __restrict__ Pd) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    { const T av = adjp[0], atv = adjtp[0];
      P[0] += av * T(1); Pd[0] += atv * T(1) + av * (T(0)); }
    { const T av = adjp[32], atv = adjtp[32];
      P[1] += av * T(1); Pd[1] += atv * T(1) + av * (T(0)); }
    { const T av = adjp[64], atv = adjtp[64];
      P[0] += av * m1_0_0; Pd[0] += atv * m1_0_0 + av * (T(1) * ux); }
    { const T av = adjp[96], atv = adjtp[96];
      P[0] += av * m0_1_0; Pd[0] += atv * m0_1_0 + av * (T(1) * uy); }
    { const T av = adjp[128], atv = adjtp[128];
      P[0] += av * m0_0_1; Pd[0] += atv * m0_0_1 + av * (T(1) * uz); }
  }
};
template <int S> struct SliceD;
template <> struct SliceD<0> {
  static constexpr int BEGIN = 0, SIZE = 5;
  template <class T> static __device__ __forceinline__ void mom(const T x, const T y, const T z, const T* __restrict__ f, T* __restrict__ acc) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    acc[0] += f[0] * T(1);
    acc[1] += f[1] * T(1);
    acc[2] += f[0] * m1_0_0;
    acc[3] += f[0] * m0_1_0;
    acc[4] += f[0] * m0_0_1;
  }
  template <class T> static __device__ __forceinline__ void grad(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T* __restrict__ adj, T& s, T& gx, T& gy, T& gz) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    { const T al = adj[0] * f[0] + adj[1] * f[1]; const T be = adj[0] * df[0] + adj[1] * df[1];
      s += be * T(1);
    }
    { const T al = adj[2] * f[0]; const T be = adj[2] * df[0];
      s += be * m1_0_0;
      gx += al * T(1);
    }
    { const T al = adj[3] * f[0]; const T be = adj[3] * df[0];
      s += be * m0_1_0;
      gy += al * T(1);
    }
    { const T al = adj[4] * f[0]; const T be = adj[4] * df[0];
      s += be * m0_0_1;
      gz += al * T(1);
    }
  }
  template <class T> static __device__ __forceinline__ void tmom(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T rdu, const T ux, const T uy, const T uz, T* __restrict__ acc) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    acc[0] += df[0] * rdu * T(1) + f[0] * (T(0));
    acc[1] += df[1] * rdu * T(1) + f[1] * (T(0));
    acc[2] += df[0] * rdu * m1_0_0 + f[0] * (T(1) * ux);
    acc[3] += df[0] * rdu * m0_1_0 + f[0] * (T(1) * uy);
    acc[4] += df[0] * rdu * m0_0_1 + f[0] * (T(1) * uz);
  }
  template <class T> static __device__ __forceinline__ void pdot(const T x, const T y, const T z, const T* __restrict__ adjp, const T* __restrict__ adjtp, const T ux, const T uy, const T uz, T* __restrict__ P, T* __restrict__ Pd) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    { const T av = adjp[0], atv = adjtp[0];
      P[0] += av * T(1); Pd[0] += atv * T(1) + av * (T(0)); }
    { const T av = adjp[32], atv = adjtp[32];
      P[1] += av * T(1); Pd[1] += atv * T(1) + av * (T(0)); }
    { const T av = adjp[64], atv = adjtp[64];
      P[0] += av * m1_0_0; Pd[0] += atv * m1_0_0 + av * (T(1) * ux); }
    { const T av = adjp[96], atv = adjtp[96];
      P[0] += av * m0_1_0; Pd[0] += atv * m0_1_0 + av * (T(1) * uy); }
    { const T av = adjp[128], atv = adjtp[128];
      P[0] += av * m0_0_1; Pd[0] += atv * m0_0_1 + av * (T(1) * uz); }
  }
};
struct Traits {
  static constexpr int L_ = L, C_ = C, V_ = V, M_ = M, NMU_ = NMU, NUMAX_ = NUMAX, NS32_ = NS32, NS64_ = NS64;
  template <int S> using F32 = SliceF<S>;
  template <int S> using F64 = SliceD<S>;
};
}  // namespace mtpgen_L6
