// Element arithmetic of the 2D Q1 finest-level operator shared by the warp-sweep kernels
// (kernels_q1.cu: one node column per lane; kernels_q1w.cu: two node columns per lane).
//
// Element product.  Writing the bilinear field of an element as
//   u = 1/4 (S + X xi + Y eta + H xi eta),  v = 1/4 (S' + X' xi + Y' eta + H' xi eta)
// with X = sum_a xi_a u_a, Y = sum_a eta_a u_a, H = sum_a xi_a eta_a u_a (xi_a, eta_a = +-1 at the
// corners) and likewise for v, the strain energy of a unit square element is
//   1/2 t^T Khat t,  t = (X, Y', G = Y + X', H, H'),
//   Khat = diag-blocks [[D11, D12], [D12, D22]]/4 on (X, Y'), D33/4 on G,
//          (D11 + D33)/12 on H, (D22 + D33)/12 on H'
// (the cross terms between constant and linear parts integrate to zero).  So K0 = T^T Khat T and
// K0 v_e costs two 4-point butterflies, 8 products and 22 multiply-adds: 37 operations instead
// of 64 multiply-adds.  The host checks T^T Khat T == K0 before using this path.
#pragma once

#include "pairs.cuh"
#include "topo_internal.cuh"

namespace topo {
namespace q1 {

template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
  using type = double2;
};
template <>
struct Vec2<float> {
  using type = float2;
};

template <typename T>
struct Q1K {
  T c11, c12, c22, c33, cH, cHp, kd;
};

template <typename T>
inline Q1K<T> coef_cast(const Q1Coef& c) {
  return Q1K<T>{(T)c.c11, (T)c.c12, (T)c.c22, (T)c.c33, (T)c.cH, (T)c.cHp, (T)c.kd};
}

// Every product and multiply-add is spelled out (no contraction left to the compiler), so that
// each kernel that calls this gives the same bits for the same inputs.
template <typename T>
__device__ __forceinline__ void q1_element(const Q1K<T>& k, T xe, const T u[4], const T v[4],
                                           T ru[4], T rv[4]) {
  const T d1 = u[2] - u[0], d2 = u[1] - u[3], s1 = u[0] + u[2], s2 = u[1] + u[3];
  const T X = d2 + d1, Y = d1 - d2, H = s1 - s2;
  const T e1 = v[2] - v[0], e2 = v[1] - v[3], t1 = v[0] + v[2], t2 = v[1] + v[3];
  const T Xp = e2 + e1, Yp = e1 - e2, Hp = t1 - t2;
  const T G = Y + Xp;
  const T a11 = mul_rn(xe, k.c11), a12 = mul_rn(xe, k.c12), a22 = mul_rn(xe, k.c22);
  const T a33 = mul_rn(xe, k.c33), aH = mul_rn(xe, k.cH), aHp = mul_rn(xe, k.cHp);
  const T gX = fma(a11, X, mul_rn(a12, Yp));
  const T gYp = fma(a12, X, mul_rn(a22, Yp));
  const T A = fma(a33, G, gX), B = fma(-a33, G, gX);
  ru[0] = fma(aH, H, -A);
  ru[1] = fma(-aH, H, B);
  ru[2] = fma(aH, H, A);
  ru[3] = fma(-aH, H, -B);
  const T C = fma(a33, G, gYp), Dd = fma(-a33, G, gYp);
  rv[0] = fma(aHp, Hp, -C);
  rv[1] = fma(-aHp, Hp, -Dd);
  rv[2] = fma(aHp, Hp, C);
  rv[3] = fma(-aHp, Hp, Dd);
}

// 1 / v rounded to nearest: the value of the IEEE division 1 / v, by the reciprocal intrinsic
// (fewer instructions than the general division sequence).
__device__ __forceinline__ float recip_rn(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double recip_rn(double v) { return __drcp_rn(v); }

template <typename T>
__device__ __forceinline__ T shfl_dn(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }

__device__ __forceinline__ double block_sum_q1(double v) {
  __shared__ double warp_sums[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) warp_sums[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// Last-block finalisation of the fused dot products of the Q1 sweeps: each block's partial sum is
// stored, and the block that arrives last sums them in block order.  DOT 1: alpha = r^T y / p^T q
// of Algorithm PCG; DOT 2: beta = r~^T y~ / r^T y.
template <int DOT>
__device__ __forceinline__ void q1_finish_dot(double part, int rhs, CgScalars* sc,
                                              double* partials, unsigned* counters) {
  const double bs = block_sum_q1(part);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[(long long)rhs * gridDim.x + blockIdx.x] = bs;
    __threadfence();
    last = (atomicAdd(&counters[rhs], 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  double s = 0.0;
  for (unsigned t = threadIdx.x; t < gridDim.x; t += blockDim.x)
    s += __ldcg(partials + (long long)rhs * gridDim.x + t);
  s = block_sum_q1(s);
  if (threadIdx.x == 0) {
    CgScalars& S = sc[rhs];
    if (DOT == 1) {
      S.pq = s;
      const double alpha = S.ry / s;
      if (!(s > 0.0) || !isfinite(alpha)) {
        S.status = TOPO_E_BREAKDOWN;
        S.done = 1;
        S.alpha = 0.0;
      } else {
        S.alpha = alpha;
      }
    } else {
      const double beta = s / S.ry;
      S.ry_new = s;
      S.beta = beta;
      S.ry = s;
      if (!isfinite(beta)) {
        S.status = TOPO_E_BREAKDOWN;
        S.done = 1;
      }
    }
    counters[rhs] = 0;
  }
}

}  // namespace q1
}  // namespace topo
