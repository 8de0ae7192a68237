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
static const unsigned fwd_ij[] = {131074u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,196611u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,262148u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,6u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u};
static const unsigned fwd_kf[] = {65541u,196614u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,5u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,131077u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,196615u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u};
static const float fwd_w[] = {1.0,1.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,1.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,1.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,1.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0};
static const unsigned adj_ij[] = {327682u,327683u,327684u,458752u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,327682u,327683u,327684u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,393216u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,393216u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,458758u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u,0u};
static const unsigned adj_kf[] = {65538u,65539u,65540u,196614u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,131074u,131075u,131076u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,65536u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,0u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,131072u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u,262144u};
static const float adj_w[] = {1.0,1.0,1.0,1.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,1.0,1.0,1.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,1.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,1.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,1.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0,0.0};
static const int fwd_layer_rows[] = {3,4};
static const int adj_layer_rows[] = {2,5};
static const int s32_begin[] = {0};
static const int s32_size[] = {5};
static const int s64_begin[] = {0};
static const int s64_size[] = {5};
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
};
struct Traits {
  static constexpr int L_ = L, C_ = C, V_ = V, M_ = M, NMU_ = NMU, NUMAX_ = NUMAX, NS32_ = NS32, NS64_ = NS64;
  template <int S> using F32 = SliceF<S>;
  template <int S> using F64 = SliceD<S>;
};
}  // namespace mtpgen_L6
