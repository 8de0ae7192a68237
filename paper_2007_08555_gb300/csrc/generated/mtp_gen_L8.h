// Generated by paper_2007_08555_gb300/codegen.py for lev_max = 8. Do not edit.
#pragma once
#include "mtp_gen_common.h"
namespace mtpgen_L8 {
constexpr int L = 8, C = 11, V = 18, M = 9, NMU = 2, NUMAX = 2;
constexpr int NS32 = 1, NS64 = 1;
constexpr int FWD_ROWS = 8, ADJ_ROWS = 10;
constexpr int FWD_LAYERS = 3, ADJ_LAYERS = 3;
constexpr int PROGRAM_OPS = 14;
constexpr int FLOP_PAIR_MOMENTS = 31, FLOP_PAIR_ADJOINT = 104, FLOP_ATOM_PROGRAM = 84;
static const int level_table[] = {9,2,1,1,0,0,4,2,1,0,0,1,0,0,6,1,1,1,0,6,1,2,0,1,0,1,1,6,3,1,0,0,1,0,0,1,0,0,8,2,1,0,0,1,1,0,8,1,2,0,2,0,2,2,8,2,1,0,0,2,0,1,0,1,1,8,4,1,0,0,1,0,0,1,0,0,1,0,0};
constexpr int LEVEL_TABLE_LEN = 79;
static const int basis_value[] = {0,13,1,11,14,15,12,16,17};
static const unsigned char comp_mu[] = {0,1,0,0,0,0,0,0,0,0,0};
static const unsigned char comp_abc[] = {0,0,0,0,0,0,1,0,0,0,1,0,0,0,1,2,0,0,1,1,0,1,0,1,0,2,0,0,1,1,0,0,2};
constexpr int NWEIGHTS = 3;
static const float weights[] = {0.0,1.0,2.0};
static const unsigned long long fwd_ops[] = {2533326330331141ull,2533322035167234ull,3096280578392064ull,3096289168392192ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,4503651167371270ull,2251847058522115ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,4503651167436807ull,2814797012008964ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2251851353817096ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,4503651167567881ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2814801307369482ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,3096284873359373ull,3096293464014848ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,3096297758261262ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull};
static const unsigned long long adj_ops[] = {2533296266018821ull,4785100374671366ull,4785104669638663ull,2533309150920712ull,4785113259573257ull,2533317740855306ull,3096229039767552ull,3096271989506048ull,3096284874473472ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2814771242729477ull,5066575351382022ull,5066579646349319ull,2814784127631368ull,5066588236283913ull,2814792717565962ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2533283381051394ull,2533287676018691ull,2533291970985988ull,3096280579309568ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2814758357762050ull,2814762652729347ull,2814766947696644ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2533274791247872ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2251799814537216ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2251799814602765ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2251799814668289ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2251799814733835ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,2814749768220686ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull,1125899906842624ull};
static const int fwd_layer_rows[] = {6,7,8};
static const int adj_layer_rows[] = {2,4,10};
static const int s32_begin[] = {0};
static const int s32_size[] = {11};
static const int s64_begin[] = {0};
static const int s64_size[] = {11};
#define MTPGEN_HAS_UNROLLED 1
template <bool WANT_B>
__device__ __forceinline__ float contract_unrolled(const float* __restrict__ src, float* __restrict__ dst, const float* __restrict__ xi, double* __restrict__ bout) {
  const float v0 = src[0];
  const float v1 = src[32];
  const float v2 = src[64];
  const float v3 = src[96];
  const float v4 = src[128];
  const float v5 = src[160];
  const float v6 = src[192];
  const float v7 = src[224];
  const float v8 = src[256];
  const float v9 = src[288];
  const float v10 = src[320];
  const float v11 = v2 * v2 + v3 * v3 + v4 * v4;
  const float v12 = v5 * v5 + 2.0f * v6 * v6 + 2.0f * v7 * v7 + v8 * v8 + 2.0f * v9 * v9 + v10 * v10;
  const float v13 = v0 * v0;
  const float v14 = v13 * v0;
  const float v15 = v0 * v1;
  const float v16 = v0 * v11;
  const float v17 = v14 * v0;
  float e = 0.f;
  e += xi[0] * v0;
  if (WANT_B) bout[0] = (double)v0;
  e += xi[1] * v13;
  if (WANT_B) bout[1] = (double)v13;
  e += xi[2] * v1;
  if (WANT_B) bout[2] = (double)v1;
  e += xi[3] * v11;
  if (WANT_B) bout[3] = (double)v11;
  e += xi[4] * v14;
  if (WANT_B) bout[4] = (double)v14;
  e += xi[5] * v15;
  if (WANT_B) bout[5] = (double)v15;
  e += xi[6] * v12;
  if (WANT_B) bout[6] = (double)v12;
  e += xi[7] * v16;
  if (WANT_B) bout[7] = (double)v16;
  e += xi[8] * v17;
  if (WANT_B) bout[8] = (double)v17;
  float a17 = xi[8];
  float a14 = xi[4];
  float a0 = xi[0];
  a14 += v0 * a17;
  a0 += v14 * a17;
  float a16 = xi[7];
  float a11 = xi[3];
  a0 += v11 * a16;
  a11 += v0 * a16;
  float a15 = xi[5];
  float a1 = xi[2];
  a0 += v1 * a15;
  a1 += v0 * a15;
  float a13 = xi[1];
  a13 += v0 * a14;
  a0 += v13 * a14;
  a0 += v0 * a13;
  a0 += v0 * a13;
  float a12 = xi[6];
  float a5 = 0.f;
  a5 += v5 * a12;
  a5 += v5 * a12;
  float a6 = 0.f;
  a6 += 2.0f * v6 * a12;
  a6 += 2.0f * v6 * a12;
  float a7 = 0.f;
  a7 += 2.0f * v7 * a12;
  a7 += 2.0f * v7 * a12;
  float a8 = 0.f;
  a8 += v8 * a12;
  a8 += v8 * a12;
  float a9 = 0.f;
  a9 += 2.0f * v9 * a12;
  a9 += 2.0f * v9 * a12;
  float a10 = 0.f;
  a10 += v10 * a12;
  a10 += v10 * a12;
  float a2 = 0.f;
  a2 += v2 * a11;
  a2 += v2 * a11;
  float a3 = 0.f;
  a3 += v3 * a11;
  a3 += v3 * a11;
  float a4 = 0.f;
  a4 += v4 * a11;
  a4 += v4 * a11;
  dst[0] = a0;
  dst[32] = a1;
  dst[64] = a2;
  dst[96] = a3;
  dst[128] = a4;
  dst[160] = a5;
  dst[192] = a6;
  dst[224] = a7;
  dst[256] = a8;
  dst[288] = a9;
  dst[320] = a10;
  return e;
}
template <int S> struct SliceF;
template <> struct SliceF<0> {
  static constexpr int BEGIN = 0, SIZE = 11;
  template <class T> static __device__ __forceinline__ void mom(const T x, const T y, const T z, const T* __restrict__ f, T* __restrict__ acc) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    const T m2_0_0 = m1_0_0 * x;
    const T m1_1_0 = m0_1_0 * x;
    const T m1_0_1 = m0_0_1 * x;
    const T m0_2_0 = m0_1_0 * y;
    const T m0_1_1 = m0_0_1 * y;
    const T m0_0_2 = m0_0_1 * z;
    acc[0] += f[0] * T(1);
    acc[1] += f[1] * T(1);
    acc[2] += f[0] * m1_0_0;
    acc[3] += f[0] * m0_1_0;
    acc[4] += f[0] * m0_0_1;
    acc[5] += f[0] * m2_0_0;
    acc[6] += f[0] * m1_1_0;
    acc[7] += f[0] * m1_0_1;
    acc[8] += f[0] * m0_2_0;
    acc[9] += f[0] * m0_1_1;
    acc[10] += f[0] * m0_0_2;
  }
  template <class T> static __device__ __forceinline__ void grad(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T* __restrict__ adj, T& s, T& gx, T& gy, T& gz) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    const T m2_0_0 = m1_0_0 * x;
    const T m1_1_0 = m0_1_0 * x;
    const T m1_0_1 = m0_0_1 * x;
    const T m0_2_0 = m0_1_0 * y;
    const T m0_1_1 = m0_0_1 * y;
    const T m0_0_2 = m0_0_1 * z;
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
    { const T al = adj[5] * f[0]; const T be = adj[5] * df[0];
      s += be * m2_0_0;
      gx += T(2) * al * m1_0_0;
    }
    { const T al = adj[6] * f[0]; const T be = adj[6] * df[0];
      s += be * m1_1_0;
      gx += al * m0_1_0;
      gy += al * m1_0_0;
    }
    { const T al = adj[7] * f[0]; const T be = adj[7] * df[0];
      s += be * m1_0_1;
      gx += al * m0_0_1;
      gz += al * m1_0_0;
    }
    { const T al = adj[8] * f[0]; const T be = adj[8] * df[0];
      s += be * m0_2_0;
      gy += T(2) * al * m0_1_0;
    }
    { const T al = adj[9] * f[0]; const T be = adj[9] * df[0];
      s += be * m0_1_1;
      gy += al * m0_0_1;
      gz += al * m0_1_0;
    }
    { const T al = adj[10] * f[0]; const T be = adj[10] * df[0];
      s += be * m0_0_2;
      gz += T(2) * al * m0_0_1;
    }
  }
  template <class T> static __device__ __forceinline__ void tmom(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T rdu, const T ux, const T uy, const T uz, T* __restrict__ acc) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    const T m2_0_0 = m1_0_0 * x;
    const T m1_1_0 = m0_1_0 * x;
    const T m1_0_1 = m0_0_1 * x;
    const T m0_2_0 = m0_1_0 * y;
    const T m0_1_1 = m0_0_1 * y;
    const T m0_0_2 = m0_0_1 * z;
    acc[0] += df[0] * rdu * T(1) + f[0] * (T(0));
    acc[1] += df[1] * rdu * T(1) + f[1] * (T(0));
    acc[2] += df[0] * rdu * m1_0_0 + f[0] * (T(1) * ux);
    acc[3] += df[0] * rdu * m0_1_0 + f[0] * (T(1) * uy);
    acc[4] += df[0] * rdu * m0_0_1 + f[0] * (T(1) * uz);
    acc[5] += df[0] * rdu * m2_0_0 + f[0] * (T(2) * m1_0_0 * ux);
    acc[6] += df[0] * rdu * m1_1_0 + f[0] * (m0_1_0 * ux + m1_0_0 * uy);
    acc[7] += df[0] * rdu * m1_0_1 + f[0] * (m0_0_1 * ux + m1_0_0 * uz);
    acc[8] += df[0] * rdu * m0_2_0 + f[0] * (T(2) * m0_1_0 * uy);
    acc[9] += df[0] * rdu * m0_1_1 + f[0] * (m0_0_1 * uy + m0_1_0 * uz);
    acc[10] += df[0] * rdu * m0_0_2 + f[0] * (T(2) * m0_0_1 * uz);
  }
  template <class T> static __device__ __forceinline__ void pdot(const T x, const T y, const T z, const T* __restrict__ adjp, const T* __restrict__ adjtp, const T ux, const T uy, const T uz, T* __restrict__ P, T* __restrict__ Pd) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    const T m2_0_0 = m1_0_0 * x;
    const T m1_1_0 = m0_1_0 * x;
    const T m1_0_1 = m0_0_1 * x;
    const T m0_2_0 = m0_1_0 * y;
    const T m0_1_1 = m0_0_1 * y;
    const T m0_0_2 = m0_0_1 * z;
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
    { const T av = adjp[160], atv = adjtp[160];
      P[0] += av * m2_0_0; Pd[0] += atv * m2_0_0 + av * (T(2) * m1_0_0 * ux); }
    { const T av = adjp[192], atv = adjtp[192];
      P[0] += av * m1_1_0; Pd[0] += atv * m1_1_0 + av * (m0_1_0 * ux + m1_0_0 * uy); }
    { const T av = adjp[224], atv = adjtp[224];
      P[0] += av * m1_0_1; Pd[0] += atv * m1_0_1 + av * (m0_0_1 * ux + m1_0_0 * uz); }
    { const T av = adjp[256], atv = adjtp[256];
      P[0] += av * m0_2_0; Pd[0] += atv * m0_2_0 + av * (T(2) * m0_1_0 * uy); }
    { const T av = adjp[288], atv = adjtp[288];
      P[0] += av * m0_1_1; Pd[0] += atv * m0_1_1 + av * (m0_0_1 * uy + m0_1_0 * uz); }
    { const T av = adjp[320], atv = adjtp[320];
      P[0] += av * m0_0_2; Pd[0] += atv * m0_0_2 + av * (T(2) * m0_0_1 * uz); }
  }
};
template <int S> struct SliceD;
template <> struct SliceD<0> {
  static constexpr int BEGIN = 0, SIZE = 11;
  template <class T> static __device__ __forceinline__ void mom(const T x, const T y, const T z, const T* __restrict__ f, T* __restrict__ acc) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    const T m2_0_0 = m1_0_0 * x;
    const T m1_1_0 = m0_1_0 * x;
    const T m1_0_1 = m0_0_1 * x;
    const T m0_2_0 = m0_1_0 * y;
    const T m0_1_1 = m0_0_1 * y;
    const T m0_0_2 = m0_0_1 * z;
    acc[0] += f[0] * T(1);
    acc[1] += f[1] * T(1);
    acc[2] += f[0] * m1_0_0;
    acc[3] += f[0] * m0_1_0;
    acc[4] += f[0] * m0_0_1;
    acc[5] += f[0] * m2_0_0;
    acc[6] += f[0] * m1_1_0;
    acc[7] += f[0] * m1_0_1;
    acc[8] += f[0] * m0_2_0;
    acc[9] += f[0] * m0_1_1;
    acc[10] += f[0] * m0_0_2;
  }
  template <class T> static __device__ __forceinline__ void grad(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T* __restrict__ adj, T& s, T& gx, T& gy, T& gz) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    const T m2_0_0 = m1_0_0 * x;
    const T m1_1_0 = m0_1_0 * x;
    const T m1_0_1 = m0_0_1 * x;
    const T m0_2_0 = m0_1_0 * y;
    const T m0_1_1 = m0_0_1 * y;
    const T m0_0_2 = m0_0_1 * z;
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
    { const T al = adj[5] * f[0]; const T be = adj[5] * df[0];
      s += be * m2_0_0;
      gx += T(2) * al * m1_0_0;
    }
    { const T al = adj[6] * f[0]; const T be = adj[6] * df[0];
      s += be * m1_1_0;
      gx += al * m0_1_0;
      gy += al * m1_0_0;
    }
    { const T al = adj[7] * f[0]; const T be = adj[7] * df[0];
      s += be * m1_0_1;
      gx += al * m0_0_1;
      gz += al * m1_0_0;
    }
    { const T al = adj[8] * f[0]; const T be = adj[8] * df[0];
      s += be * m0_2_0;
      gy += T(2) * al * m0_1_0;
    }
    { const T al = adj[9] * f[0]; const T be = adj[9] * df[0];
      s += be * m0_1_1;
      gy += al * m0_0_1;
      gz += al * m0_1_0;
    }
    { const T al = adj[10] * f[0]; const T be = adj[10] * df[0];
      s += be * m0_0_2;
      gz += T(2) * al * m0_0_1;
    }
  }
  template <class T> static __device__ __forceinline__ void tmom(const T x, const T y, const T z, const T* __restrict__ f, const T* __restrict__ df, const T rdu, const T ux, const T uy, const T uz, T* __restrict__ acc) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    const T m2_0_0 = m1_0_0 * x;
    const T m1_1_0 = m0_1_0 * x;
    const T m1_0_1 = m0_0_1 * x;
    const T m0_2_0 = m0_1_0 * y;
    const T m0_1_1 = m0_0_1 * y;
    const T m0_0_2 = m0_0_1 * z;
    acc[0] += df[0] * rdu * T(1) + f[0] * (T(0));
    acc[1] += df[1] * rdu * T(1) + f[1] * (T(0));
    acc[2] += df[0] * rdu * m1_0_0 + f[0] * (T(1) * ux);
    acc[3] += df[0] * rdu * m0_1_0 + f[0] * (T(1) * uy);
    acc[4] += df[0] * rdu * m0_0_1 + f[0] * (T(1) * uz);
    acc[5] += df[0] * rdu * m2_0_0 + f[0] * (T(2) * m1_0_0 * ux);
    acc[6] += df[0] * rdu * m1_1_0 + f[0] * (m0_1_0 * ux + m1_0_0 * uy);
    acc[7] += df[0] * rdu * m1_0_1 + f[0] * (m0_0_1 * ux + m1_0_0 * uz);
    acc[8] += df[0] * rdu * m0_2_0 + f[0] * (T(2) * m0_1_0 * uy);
    acc[9] += df[0] * rdu * m0_1_1 + f[0] * (m0_0_1 * uy + m0_1_0 * uz);
    acc[10] += df[0] * rdu * m0_0_2 + f[0] * (T(2) * m0_0_1 * uz);
  }
  template <class T> static __device__ __forceinline__ void pdot(const T x, const T y, const T z, const T* __restrict__ adjp, const T* __restrict__ adjtp, const T ux, const T uy, const T uz, T* __restrict__ P, T* __restrict__ Pd) {
    const T m1_0_0 = x;
    const T m0_1_0 = y;
    const T m0_0_1 = z;
    const T m2_0_0 = m1_0_0 * x;
    const T m1_1_0 = m0_1_0 * x;
    const T m1_0_1 = m0_0_1 * x;
    const T m0_2_0 = m0_1_0 * y;
    const T m0_1_1 = m0_0_1 * y;
    const T m0_0_2 = m0_0_1 * z;
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
    { const T av = adjp[160], atv = adjtp[160];
      P[0] += av * m2_0_0; Pd[0] += atv * m2_0_0 + av * (T(2) * m1_0_0 * ux); }
    { const T av = adjp[192], atv = adjtp[192];
      P[0] += av * m1_1_0; Pd[0] += atv * m1_1_0 + av * (m0_1_0 * ux + m1_0_0 * uy); }
    { const T av = adjp[224], atv = adjtp[224];
      P[0] += av * m1_0_1; Pd[0] += atv * m1_0_1 + av * (m0_0_1 * ux + m1_0_0 * uz); }
    { const T av = adjp[256], atv = adjtp[256];
      P[0] += av * m0_2_0; Pd[0] += atv * m0_2_0 + av * (T(2) * m0_1_0 * uy); }
    { const T av = adjp[288], atv = adjtp[288];
      P[0] += av * m0_1_1; Pd[0] += atv * m0_1_1 + av * (m0_0_1 * uy + m0_1_0 * uz); }
    { const T av = adjp[320], atv = adjtp[320];
      P[0] += av * m0_0_2; Pd[0] += atv * m0_0_2 + av * (T(2) * m0_0_1 * uz); }
  }
};
struct Traits {
  static constexpr int L_ = L, C_ = C, V_ = V, M_ = M, NMU_ = NMU, NUMAX_ = NUMAX, NS32_ = NS32, NS64_ = NS64;
  template <int S> using F32 = SliceF<S>;
  template <int S> using F64 = SliceD<S>;
};
}  // namespace mtpgen_L8
