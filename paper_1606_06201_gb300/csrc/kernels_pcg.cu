// Vector kernels of Algorithm PCG (Sec. 5.2) in FP64 with the paper's sign convention
// r = A z - b, p = -y:  alpha = r^T y / p^T A p,  z += alpha p,  r~ = r + alpha A p,
// beta = r~^T y~ / r^T y,  p = -y~ + beta p.  Stop test ||r||_2 / ||b||_2 <= tol.
//
// Every reduction is a fixed-grid grid-stride kernel writing one partial per block; the last
// block to finish (atomic ticket) adds the partials in block order, so sums are deterministic,
// and updates the device-resident scalars of its right-hand side.  Kernels return at once for a
// right-hand side whose recurrence has stopped, which lets a captured graph of several
// iterations run past convergence at the cost of empty launches.
#include "pairs.cuh"
#include "topo_internal.cuh"

namespace topo {

namespace {

__device__ __forceinline__ double block_sum(double v) {
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

// Writes this block's partials (NV values) and returns true in the whole block of the last block
// to finish; the sums are then returned in tot[] (valid in every thread of that block).
template <int NV>
__device__ bool last_block_sums(const double (&part)[NV], double* partials, unsigned* counters,
                                int rhs, double (&tot)[NV]) {
  static_assert(NV <= kMaxRedValues, "partials buffers hold kMaxRedValues values per block");
  __shared__ bool last;
  __shared__ double res[NV];
  double bs[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) bs[q] = block_sum(part[q]);
  const long long base = (long long)rhs * gridDim.x * NV;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[base + (long long)q * gridDim.x + blockIdx.x] = bs[q];
    __threadfence();
    last = (atomicAdd(&counters[rhs], 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = 0.0;
    for (unsigned t = threadIdx.x; t < gridDim.x; t += blockDim.x)
      s += __ldcg(partials + base + (long long)q * gridDim.x + t);
    s = block_sum(s);
    if (threadIdx.x == 0) res[q] = s;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) tot[q] = res[q];
  if (threadIdx.x == 0) counters[rhs] = 0;
  return true;
}

// The per-iteration vector kernels move two elements per 16-byte access (a grid-stride loop over
// single doubles left each warp one 8-byte load per vector in flight: 37% of the copy bandwidth
// in k_cg_update).  The pair path needs n even and
// every vector of the right-hand side 16-byte aligned (8-byte for the FP32 copies); otherwise the
// single-element loop runs.  Either way the sums are taken in a fixed order per grid shape.
template <typename TV>
struct Pair2;
template <>
struct Pair2<double> {
  using type = double2;
};
template <>
struct Pair2<float> {
  using type = float2;
};

__device__ __forceinline__ bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
__device__ __forceinline__ bool al8(const void* p) { return ((uintptr_t)p & 7u) == 0; }
template <typename TV>
__device__ __forceinline__ bool al_pair(const TV* p) {
  return sizeof(TV) == 8 ? al16(p) : al8(p);
}

// r = A z0 - b (use_x0) or r = -b, z = 0; ||b||, ||r|| -> initial scalars and stop test.
// CG scalars at the start: ||b||, r^T r and the stop test of Algorithm PCG on them.
__device__ __forceinline__ CgScalars cg_start_scalars(double bb, double rr, double tol,
                                                      int max_iter) {
  CgScalars S = {};
  S.bnorm = sqrt(bb);
  S.rr = rr;
  S.rel = S.bnorm > 0.0 ? sqrt(rr) / S.bnorm : 0.0;
  S.iter = 0;
  S.status = TOPO_OK;
  if (!isfinite(S.rel)) {
    S.status = TOPO_E_BREAKDOWN;
    S.done = 1;
  } else {
    S.done = (S.bnorm == 0.0 || S.rel <= tol) ? 1 : 0;
    if (!S.done && max_iter <= 0) {
      S.done = 1;
      S.status = TOPO_E_NOT_CONVERGED;
    }
  }
  return S;
}

__global__ void __launch_bounds__(kThreads) k_cg_init(long long n, const double* __restrict__ b,
                                                      double* __restrict__ z,
                                                      double* __restrict__ r,
                                                      const double* __restrict__ Az, int use_x0,
                                                      double* partials, unsigned* counters,
                                                      CgScalars* sc, double tol, int max_iter) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  b += rhs * n;
  z += rhs * n;
  r += rhs * n;
  if (Az) Az += rhs * n;
  double part[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double bi = b[i];
    const double ri = use_x0 ? Az[i] - bi : -bi;
    if (!use_x0) z[i] = 0.0;
    r[i] = ri;
    part[0] = fma(bi, bi, part[0]);
    part[1] = fma(ri, ri, part[1]);
  }
  double tot[2];
  if (!last_block_sums<2>(part, partials, counters, rhs, tot)) return;
  if (threadIdx.x == 0) sc[rhs] = cg_start_scalars(tot[0], tot[1], tol, max_iter);
}

// The same from the caller's right-hand side with zero start (use_x0 = 0) in one pass: b masked
// on fixed DOFs (index < n_mask), z = 0, r = -b, and the FP32 copy of r for the V-cycle (rv, or
// none): the values of k_mask_copy, k_cg_init and k_d2f in sequence.
template <typename TV>
__global__ void __launch_bounds__(kThreads) k_cg_init_zero(long long n, long long n_mask,
                                                           const double* __restrict__ b,
                                                           const uint8_t* __restrict__ fixed,
                                                           double* __restrict__ z,
                                                           double* __restrict__ r,
                                                           TV* __restrict__ rv, double* partials,
                                                           unsigned* counters, CgScalars* sc,
                                                           double tol, int max_iter) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  b += rhs * n;
  z += rhs * n;
  r += rhs * n;
  if (rv) rv += rhs * n;
  double part[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double bi = (i < n_mask && fixed[i]) ? 0.0 : b[i];
    const double ri = -bi;
    z[i] = 0.0;
    r[i] = ri;
    if (rv) rv[i] = tv_from_double<TV>(ri);
    part[0] = fma(bi, bi, part[0]);
    part[1] = fma(ri, ri, part[1]);
  }
  double tot[2];
  if (!last_block_sums<2>(part, partials, counters, rhs, tot)) return;
  if (threadIdx.x == 0) sc[rhs] = cg_start_scalars(tot[0], tot[1], tol, max_iter);
}

// p = -y (first direction), y_old = y, and r^T y.
template <typename TV>
__global__ void __launch_bounds__(kThreads) k_cg_start_p(long long n, const double* __restrict__ r,
                                                         const TV* __restrict__ y,
                                                         double* __restrict__ p,
                                                         TV* __restrict__ y_old, int flexible,
                                                         double* partials, unsigned* counters,
                                                         CgScalars* sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc[rhs].done) return;
  r += rhs * n;
  y += rhs * n;
  p += rhs * n;
  if (flexible) y_old += rhs * n;
  double part[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const TV yi = y[i];
    p[i] = -double_of(yi);
    if (flexible) y_old[i] = yi;
    part[0] = fma(r[i], double_of(yi), part[0]);
  }
  double tot[1];
  if (!last_block_sums<1>(part, partials, counters, rhs, tot)) return;
  if (threadIdx.x == 0) {
    sc[rhs].ry = tot[0];
    if (!isfinite(tot[0])) {
      sc[rhs].status = TOPO_E_BREAKDOWN;
      sc[rhs].done = 1;
    }
  }
}

// z += alpha p, r += alpha q, rv = r (V-cycle input precision), ||r||^2 and the stop test.
template <typename TV>
// (z += alpha p of this iteration is applied by k_cg_p, which reads p anyway, or by
// k_cg_finish_z when the iteration ends the solve.)
__global__ void __launch_bounds__(kThreads, 4) k_cg_update(long long n, double* __restrict__ z,
                                                        double* __restrict__ r,
                                                        const double* __restrict__ p,
                                                        const double* __restrict__ q,
                                                        TV* __restrict__ rv, double* partials,
                                                        unsigned* counters, CgScalars* sc,
                                                        double tol, int max_iter) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc[rhs].done) return;
  const double alpha = sc[rhs].alpha;
  z += rhs * n;
  r += rhs * n;
  p += rhs * n;
  q += rhs * n;
  if (rv) rv += rhs * n;
  double part[1] = {0.0};
  // Mixed solver: ||r|| serves the stop test only, and is formed from the FP32 copy of r scaled
  // by 1 / ||b|| (FP32 squares summed per thread; relative error about 1e-6 for the few dozen
  // entries a thread takes), so that the update is the only FP64 multiply-add per DOF.
  const double inv_bn = 1.0 / sc[rhs].bnorm;
  const bool f32norm = sizeof(TV) == 4 && rv && inv_bn >= 1e-30 && inv_bn <= 1e30;
  const float sinv = f32norm ? float_from_double_rn(inv_bn) : 0.0f;
  float partf = 0.0f;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  if ((n & 1) == 0 && al16(r) && al16(q) && (!rv || al_pair(rv))) {
    using V2 = typename Pair2<TV>::type;
    const long long np = n >> 1;
    double2* __restrict__ r2 = reinterpret_cast<double2*>(r);
    const double2* __restrict__ q2 = reinterpret_cast<const double2*>(q);
    V2* __restrict__ rv2 = reinterpret_cast<V2*>(rv);
    auto put = [&](int j, double2 sa) {
      r2[j] = sa;
      if (rv) {
        V2 va;
        va.x = tv_from_double<TV>(sa.x);
        va.y = tv_from_double<TV>(sa.y);
        rv2[j] = va;
        if constexpr (sizeof(TV) == 4) {
          if (f32norm) {
            const float ux = va.x * sinv, uy = va.y * sinv;
            partf = fmaf(ux, ux, partf);
            partf = fmaf(uy, uy, partf);
            return;
          }
        }
      }
      part[0] = fma(sa.x, sa.x, part[0]);
      part[0] = fma(sa.y, sa.y, part[0]);
    };
    const int npi = (int)np, nti = (int)nt;  // (fewer than 2^31 entries)
    int j = (int)t0;
    // four pairs' loads before any store (the fixed reduction grid keeps half the warps
    // resident, so each thread keeps more bytes in flight)
    for (; j + 3 * nti < npi; j += 4 * nti) {
      double2 qv[4], rv4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        qv[u] = q2[j + u * nti];
        rv4[u] = r2[j + u * nti];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        put(j + u * nti, make_double2(fma(alpha, qv[u].x, rv4[u].x), fma(alpha, qv[u].y, rv4[u].y)));
    }
    for (; j < npi; j += nti) {
      const double2 qa = q2[j], ra = r2[j];
      put(j, make_double2(fma(alpha, qa.x, ra.x), fma(alpha, qa.y, ra.y)));
    }
  } else {  // (odd n, e.g. 3D grids, or unaligned vectors)
    auto put1 = [&](long long i, double ri) {
      r[i] = ri;
      if (rv) {
        const TV vi = tv_from_double<TV>(ri);
        rv[i] = vi;
        if constexpr (sizeof(TV) == 4) {
          if (f32norm) {
            const float ui = vi * sinv;
            partf = fmaf(ui, ui, partf);
            return;
          }
        }
      }
      part[0] = fma(ri, ri, part[0]);
    };
    long long i = t0;
    // three entries' loads before any store, the sums in the same order as one at a time
    for (; i + 2 * nt < n; i += 3 * nt) {
      double qv[3], r0[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        qv[u] = q[i + u * nt];
        r0[u] = r[i + u * nt];
      }
#pragma unroll
      for (int u = 0; u < 3; ++u) put1(i + u * nt, fma(alpha, qv[u], r0[u]));
    }
    for (; i < n; i += nt) put1(i, fma(alpha, q[i], r[i]));
  }
  if (f32norm) part[0] = (double)partf;
  double tot[1];
  if (!last_block_sums<1>(part, partials, counters, rhs, tot)) return;
  if (threadIdx.x == 0) {
    CgScalars& S = sc[rhs];
    S.rr = f32norm ? tot[0] * S.bnorm * S.bnorm : tot[0];
    S.rel = f32norm ? sqrt(tot[0]) : sqrt(tot[0]) / S.bnorm;
    S.iter += 1;
    if (!isfinite(S.rel)) {
      S.status = TOPO_E_BREAKDOWN;
      S.done = 1;
    } else if (S.rel <= tol) {
      S.done = 1;
    } else if (S.iter >= max_iter) {
      S.status = TOPO_E_NOT_CONVERGED;
      S.done = 1;
    }
  }
}

// beta = r~^T y~ / r^T y (flexible: (r~^T y~ - r~^T y) / r^T y).
template <typename TV>
__global__ void __launch_bounds__(kThreads) k_cg_beta(long long n, const double* __restrict__ r,
                                                      const TV* __restrict__ y,
                                                      const TV* __restrict__ y_old, int flexible,
                                                      double* partials, unsigned* counters,
                                                      CgScalars* sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc[rhs].done) return;
  r += rhs * n;
  y += rhs * n;
  if (flexible) y_old += rhs * n;
  double part[2] = {0.0, 0.0};
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  if ((n & 1) == 0 && al16(r) && al_pair(y) && (!flexible || al_pair(y_old))) {
    using V2 = typename Pair2<TV>::type;
    const long long np = n >> 1;
    const double2* __restrict__ r2 = reinterpret_cast<const double2*>(r);
    const V2* __restrict__ y2 = reinterpret_cast<const V2*>(y);
    const V2* __restrict__ yo2 = reinterpret_cast<const V2*>(y_old);
    for (long long j = t0; j < np; j += nt) {
      const double2 rr = r2[j];
      const V2 yv = y2[j];
      part[0] = fma(rr.x, double_of(yv.x), part[0]);
      part[0] = fma(rr.y, double_of(yv.y), part[0]);
      if (flexible) {
        const V2 yo = yo2[j];
        part[1] = fma(rr.x, double_of(yo.x), part[1]);
        part[1] = fma(rr.y, double_of(yo.y), part[1]);
      }
    }
  } else {
    for (long long i = t0; i < n; i += nt) {
      const double ri = r[i];
      part[0] = fma(ri, double_of(y[i]), part[0]);
      if (flexible) part[1] = fma(ri, double_of(y_old[i]), part[1]);
    }
  }
  double tot[2];
  if (!last_block_sums<2>(part, partials, counters, rhs, tot)) return;
  if (threadIdx.x == 0) {
    CgScalars& S = sc[rhs];
    const double num = flexible ? tot[0] - tot[1] : tot[0];
    const double beta = num / S.ry;
    S.ry_new = tot[0];
    S.ry_old = tot[1];
    S.beta = beta;
    S.ry = tot[0];
    if (!isfinite(beta)) {
      S.status = TOPO_E_BREAKDOWN;
      S.done = 1;
    }
  }
}

// z += alpha p (the iterate update of the iteration now ending), then p = -y + beta p, y_old = y.
// (Scalar accesses: a version with 16-byte accesses, two pairs per iteration, measured 26.6 us
// against 19.3 us at 4.2M DOFs; three entries' loads in flight per thread made the 2048 x 1024 step
// 4.584 against 4.567 ms.)
template <typename TV>
__global__ void __launch_bounds__(kThreads) k_cg_p(long long n, const TV* __restrict__ y,
                                                   double* __restrict__ p, TV* __restrict__ y_old,
                                                   int flexible, const CgScalars* sc,
                                                   double* __restrict__ z) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc[rhs].done) return;
  const double beta = sc[rhs].beta, alpha = sc[rhs].alpha;
  y += rhs * n;
  p += rhs * n;
  z += rhs * n;
  if (flexible) y_old += rhs * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const TV yi = y[i];
    const double pi = p[i];
    z[i] = fma(alpha, pi, z[i]);
    p[i] = fma(beta, pi, -(double)yi);  // (the hardware widening: 19.3 against 23.3 us here)
    if (flexible) y_old[i] = yi;
  }
}

// The iterate update of the iteration that ended the solve (its direction update did not run):
// z += alpha p for every right-hand side with alpha != 0 (alpha = 0: stopped before an update,
// or a breakdown in the operator).
__global__ void __launch_bounds__(kThreads) k_cg_finish_z(long long n, const double* __restrict__ p,
                                                          double* __restrict__ z,
                                                          const CgScalars* sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  const double alpha = sc[rhs].alpha;
  if (alpha == 0.0) return;
  p += rhs * n;
  z += rhs * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    z[i] = fma(alpha, p[i], z[i]);
}

__global__ void __launch_bounds__(kThreads) k_dot(long long n, const double* __restrict__ a,
                                                  const double* __restrict__ b, double* partials,
                                                  unsigned* counters, double* out) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  a += rhs * n;
  b += rhs * n;
  double part[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    part[0] = fma(a[i], b[i], part[0]);
  double tot[1];
  if (!last_block_sums<1>(part, partials, counters, rhs, tot)) return;
  if (threadIdx.x == 0) out[rhs] = tot[0];
}

__global__ void __launch_bounds__(kThreads) k_cg_alpha(long long n, const double* __restrict__ p,
                                                       const double* __restrict__ q,
                                                       double* partials, unsigned* counters,
                                                       CgScalars* sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc[rhs].done) return;
  p += rhs * n;
  q += rhs * n;
  double part[1] = {0.0};
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  if ((n & 1) == 0 && al16(p) && al16(q)) {
    const long long np = n >> 1;
    const double2* __restrict__ p2 = reinterpret_cast<const double2*>(p);
    const double2* __restrict__ q2 = reinterpret_cast<const double2*>(q);
    for (long long j = t0; j < np; j += nt) {
      const double2 pa = p2[j], qa = q2[j];
      part[0] = fma(pa.x, qa.x, part[0]);
      part[0] = fma(pa.y, qa.y, part[0]);
    }
  } else {
    for (long long i = t0; i < n; i += nt) part[0] = fma(p[i], q[i], part[0]);
  }
  double tot[1];
  if (!last_block_sums<1>(part, partials, counters, rhs, tot)) return;
  if (threadIdx.x == 0) {
    CgScalars& S = sc[rhs];
    S.pq = tot[0];
    const double alpha = S.ry / tot[0];
    if (!(tot[0] > 0.0) || !isfinite(alpha)) {
      S.status = TOPO_E_BREAKDOWN;
      S.done = 1;
      S.alpha = 0.0;
    } else {
      S.alpha = alpha;
    }
  }
}

// dst = src with the fixed DOFs zeroed (n_mask DOFs carry a mask; entries beyond it, such as the
// lambda entry of an IP system, are copied unchanged).
__global__ void k_mask_copy(long long n, long long n_mask, const double* __restrict__ src,
                            double* __restrict__ dst, const uint8_t* __restrict__ fixed) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  src += rhs * n;
  dst += rhs * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (i < n_mask && fixed[i]) ? 0.0 : src[i];
}

// ---- largest eigenvalue of D^{-1} A by power iteration (per-level Jacobi damping) ----------
// v0: a fixed pseudo-random vector (integer hash of the index), zero on fixed DOFs.
__global__ void k_power_init(long long n, int arrow, double* v, const uint8_t* fixed) {
  pdl_prologue();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    unsigned h = (unsigned)(i * 2654435761ull) ^ 0x9e3779b9u;
    h ^= h >> 15;
    h *= 0x2c1b3c6du;
    h ^= h >> 12;
    v[i] = fixed[i] ? 0.0 : 0.5 + (double)(h & 0xffffu) / 65536.0;
  }
  if (arrow && i == 0) v[n] = 1.0;
}

// w = D^{-1} y; partial sums of v^T y, v^T D v, w^T D w (D = 1/invd; lambda entry D = zll);
// last block: est[0] = Rayleigh quotient v^T A v / v^T D v, est[1] = 1/||w||_D.
__global__ void __launch_bounds__(kThreads) k_power_step(long long n, int arrow,
                                                         const double* __restrict__ v,
                                                         const double* __restrict__ y,
                                                         const double* __restrict__ invd,
                                                         const double* zll, double* __restrict__ w,
                                                         double* partials, unsigned* counters,
                                                         double* est) {
  pdl_prologue();
  double part[3] = {0.0, 0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double vi = v[i], yi = y[i], di = invd[i];
    const double wi = di * yi;
    w[i] = wi;
    part[0] = fma(vi, yi, part[0]);
    part[1] = fma(vi, vi / di, part[1]);
    part[2] = fma(wi, wi / di, part[2]);
  }
  if (arrow && blockIdx.x == 0 && threadIdx.x == 0) {
    const double z = *zll, vi = v[n], yi = y[n], wi = yi / z;
    w[n] = wi;
    part[0] = fma(vi, yi, part[0]);
    part[1] = fma(vi, vi * z, part[1]);
    part[2] = fma(wi, wi * z, part[2]);
  }
  double tot[3];
  if (!last_block_sums<3>(part, partials, counters, 0, tot)) return;
  if (threadIdx.x == 0) {
    est[0] = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
    est[1] = tot[2] > 0.0 ? 1.0 / sqrt(tot[2]) : 0.0;
  }
}

__global__ void k_power_scale(long long n, const double* __restrict__ w, double* __restrict__ v,
                              const double* est) {
  pdl_prologue();
  const double sc = est[1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = w[i] * sc;
}

__global__ void k_power_store(const double* est, double* lam_dev) {
  pdl_prologue();
  if (threadIdx.x == 0 && blockIdx.x == 0) *lam_dev = est[0];
}

// omega_k = min(omega, c / (1.05 lambda)); invd <- omega_k invd.
__global__ void k_power_finish(long long n, const double* est, double omega, double c,
                               double* omega_dev, double* invd) {
  pdl_prologue();
  const double lam = est[0];
  const double om = lam > 0.0 ? fmin(omega, c / (1.05 * lam)) : omega;
  if (blockIdx.x == 0 && threadIdx.x == 0) *omega_dev = om;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    invd[i] *= om;
}

// One step of the Chebyshev smoother on D^{-1} A over [lam/alpha, 1.05 lam] (lam from the power
// iteration): theta = (a+b)/2, delta = (b-a)/2, sigma = theta/delta, rho_0 = 1/sigma,
// rho_j = 1/(2 sigma - rho_{j-1});  d_0 = D^{-1} t / theta,
// d_j = rho_j rho_{j-1} d_{j-1} + (2 rho_j / delta) D^{-1} t;  z += d_j;  t = b - A z.
template <typename T>
__global__ void k_cheb_update(long long n, int step, int z_zero, const double* lam_dev,
                              double alpha, const T* __restrict__ invd, const T* __restrict__ t,
                              T* __restrict__ d, T* __restrict__ z,
                              const uint8_t* __restrict__ fixed, const CgScalars* sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const double lam = *lam_dev;
  const double b = 1.05 * lam, a = lam / alpha;
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
  double rho_prev = 1.0 / sigma, rho = rho_prev;
  for (int j = 1; j <= step; ++j) {
    rho_prev = rho;
    rho = 1.0 / (2.0 * sigma - rho_prev);
  }
  const T c_old = step == 0 ? T(0) : (T)(rho * rho_prev);
  const T c_new = step == 0 ? (T)(1.0 / theta) : (T)(2.0 * rho / delta);
  t += rhs * n;
  d += rhs * n;
  z += rhs * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (fixed[i]) {
      if (z_zero) z[i] = T(0);
      continue;
    }
    const T di = (step == 0 ? T(0) : c_old * d[i]) + c_new * invd[i] * t[i];
    d[i] = di;
    z[i] = z_zero ? di : z[i] + di;
  }
}

// Loop control of the persistent CG graph: keep iterating while any right-hand side runs.
// The iteration count bounds the loop even if a right-hand side were never marked done.
__global__ void k_loop_cond(cudaGraphConditionalHandle handle, const CgScalars* sc, int nrhs,
                            int max_iter) {
  pdl_prologue();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned running = 0;
  for (int k = 0; k < nrhs; ++k) running |= (!sc[k].done && sc[k].iter < max_iter) ? 1u : 0u;
  cudaGraphSetConditional(handle, running);
}

inline unsigned red_blocks(long long n) {
  const long long b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b < kRedBlocks ? (b < 1 ? 1 : b) : kRedBlocks);
}

// Self-check of the integer conversions of pairs.cuh against the hardware conversions: counts
// the inputs whose results differ (bad[0]: double -> float, bad[1]: float -> double; two NaNs
// count as equal).
__global__ void k_check_conversions(const double* __restrict__ d, const float* __restrict__ f,
                                    long long n, unsigned long long* bad) {
  unsigned long long b0 = 0, b1 = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float a = float_from_double_rn(d[i]), h = __double2float_rn(d[i]);
    if (!((a != a && h != h) || __float_as_uint(a) == __float_as_uint(h))) ++b0;
    const double c = double_from_float_exact(f[i]), e = (double)f[i];
    if (!((c != c && e != e) || __double_as_longlong(c) == __double_as_longlong(e))) ++b1;
  }
  if (b0) atomicAdd(bad, b0);
  if (b1) atomicAdd(bad + 1, b1);
}

}  // namespace

cudaError_t launch_cg_init(long long n, int nrhs, const double* b, double* z, double* r,
                           const double* Az, int use_x0, double* partials, unsigned* counters,
                           CgScalars* sc, double tol, int max_iter, cudaStream_t st) {
  topo::launch(k_cg_init, dim3(red_blocks(n), nrhs), kThreads, 0, st, n, b, z, r, Az, use_x0, partials,
                                                            counters, sc, tol, max_iter);
  return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_cg_init_zero(long long n, long long n_mask, int nrhs, const double* b,
                                const uint8_t* fixed, double* z, double* r, TV* rv,
                                double* partials, unsigned* counters, CgScalars* sc, double tol,
                                int max_iter, cudaStream_t st) {
  topo::launch(k_cg_init_zero<TV>, dim3(red_blocks(n), nrhs), kThreads, 0, st, n, n_mask, b, fixed,
               z, r, rv, partials, counters, sc, tol, max_iter);
  return cudaGetLastError();
}
template cudaError_t launch_cg_init_zero<float>(long long, long long, int, const double*,
                                                const uint8_t*, double*, double*, float*, double*,
                                                unsigned*, CgScalars*, double, int, cudaStream_t);
template cudaError_t launch_cg_init_zero<double>(long long, long long, int, const double*,
                                                 const uint8_t*, double*, double*, double*,
                                                 double*, unsigned*, CgScalars*, double, int,
                                                 cudaStream_t);

template <typename TV>
cudaError_t launch_cg_start_p(long long n, int nrhs, const double* r, const TV* y, double* p,
                              TV* y_old, int flexible, double* partials, unsigned* counters,
                              CgScalars* sc, cudaStream_t st) {
  topo::launch(k_cg_start_p<TV>, dim3(red_blocks(n), nrhs), kThreads, 0, st, n, r, y, p, y_old, flexible,
                                                                   partials, counters, sc);
  return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_cg_update(long long n, int nrhs, double* z, double* r, const double* p,
                             const double* q, TV* rv, double* partials, unsigned* counters,
                             CgScalars* sc, double tol, int max_iter, cudaStream_t st) {
  topo::launch(k_cg_update<TV>, dim3(red_blocks(n), nrhs), kThreads, 0, st, n, z, r, p, q, rv, partials,
                                                                  counters, sc, tol, max_iter);
  return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_cg_direction(long long n, int nrhs, const double* r, const TV* y, double* p,
                                TV* y_old, int flexible, double* partials, unsigned* counters,
                                CgScalars* sc, cudaStream_t st, double* z) {
  topo::launch(k_cg_beta<TV>, dim3(red_blocks(n), nrhs), kThreads, 0, st, n, r, y, y_old, flexible,
                                                                partials, counters, sc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  topo::launch(k_cg_p<TV>, dim3(red_blocks(n), nrhs), kThreads, 0, st, n, y, p, y_old, flexible, sc,
               z);
  return cudaGetLastError();
}

cudaError_t launch_cg_finish_z(long long n, int nrhs, const double* p, double* z,
                               const CgScalars* sc, cudaStream_t st) {
  topo::launch(k_cg_finish_z, dim3(red_blocks(n), nrhs), kThreads, 0, st, n, p, z, sc);
  return cudaGetLastError();
}

cudaError_t launch_power_init(long long n, int arrow, double* v, const uint8_t* fixed,
                              cudaStream_t st) {
  topo::launch(k_power_init, blocks_for(n), kThreads, 0, st, n, arrow, v, fixed);
  return cudaGetLastError();
}

cudaError_t launch_power_step(long long n, int arrow, const double* v, const double* y,
                              const double* invd, const double* zll, double* w, double* partials,
                              unsigned* counters, double* est, cudaStream_t st) {
  topo::launch(k_power_step, red_blocks(n), kThreads, 0, st, n, arrow, v, y, invd, zll, w, partials,
                                                   counters, est);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  topo::launch(k_power_scale, red_blocks(n + arrow), kThreads, 0, st, n + arrow, w, (double*)v, est);
  return cudaGetLastError();
}

cudaError_t launch_power_store(const double* est, double* lam_dev, cudaStream_t st) {
  topo::launch(k_power_store, 1, 32, 0, st, est, lam_dev);
  return cudaGetLastError();
}

cudaError_t launch_power_finish(long long n, const double* est, double omega, double c,
                                double* omega_dev, double* invd, cudaStream_t st) {
  topo::launch(k_power_finish, red_blocks(n), kThreads, 0, st, n, est, omega, c, omega_dev, invd);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cheb_update(long long n, int nrhs, int step, int z_zero, const double* lam_dev,
                               double alpha, const T* invd, const T* t, T* d, T* z,
                               const uint8_t* fixed, const CgScalars* sc, cudaStream_t st) {
  topo::launch(k_cheb_update<T>, dim3(blocks_for(n), nrhs), kThreads, 0, st, n, step, z_zero,
               lam_dev, alpha, invd, t, d, z, fixed, sc);
  return cudaGetLastError();
}
template cudaError_t launch_cheb_update<double>(long long, int, int, int, const double*, double,
                                                const double*, const double*, double*, double*,
                                                const uint8_t*, const CgScalars*, cudaStream_t);
template cudaError_t launch_cheb_update<float>(long long, int, int, int, const double*, double,
                                               const float*, const float*, float*, float*,
                                               const uint8_t*, const CgScalars*, cudaStream_t);

cudaError_t launch_power_store(const double* est, double* lam_dev, cudaStream_t st);

cudaError_t launch_loop_cond(cudaGraphConditionalHandle handle, const CgScalars* sc, int nrhs,
                             int max_iter, cudaStream_t st) {
  topo::launch(k_loop_cond, 1, 32, 0, st, handle, sc, nrhs, max_iter);
  return cudaGetLastError();
}

cudaError_t launch_mask_copy(long long n, long long n_mask, int nrhs, const double* src,
                             double* dst, const uint8_t* fixed, cudaStream_t st) {
  topo::launch(k_mask_copy, dim3(red_blocks(n), nrhs), kThreads, 0, st, n, n_mask, src, dst, fixed);
  return cudaGetLastError();
}

cudaError_t launch_cg_alpha(long long n, int nrhs, const double* p, const double* q,
                            double* partials, unsigned* counters, CgScalars* sc, cudaStream_t st) {
  topo::launch(k_cg_alpha, dim3(red_blocks(n), nrhs), kThreads, 0, st, n, p, q, partials, counters, sc);
  return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_cg_p(long long n, int nrhs, const TV* y, double* p, TV* y_old, int flexible,
                        CgScalars* sc, cudaStream_t st, double* z) {
  topo::launch(k_cg_p<TV>, dim3(red_blocks(n), nrhs), kThreads, 0, st, n, y, p, y_old, flexible, sc,
               z);
  return cudaGetLastError();
}
template cudaError_t launch_cg_p<double>(long long, int, const double*, double*, double*, int,
                                         CgScalars*, cudaStream_t, double*);
template cudaError_t launch_cg_p<float>(long long, int, const float*, double*, float*, int,
                                        CgScalars*, cudaStream_t, double*);

cudaError_t launch_dot(long long n, int nrhs, const double* a, const double* b, double* partials,
                       unsigned* counters, double* out, cudaStream_t st) {
  topo::launch(k_dot, dim3(red_blocks(n), nrhs), kThreads, 0, st, n, a, b, partials, counters, out);
  return cudaGetLastError();
}

#define TOPO_INST(TV)                                                                            \
  template cudaError_t launch_cg_start_p<TV>(long long, int, const double*, const TV*, double*,  \
                                             TV*, int, double*, unsigned*, CgScalars*,           \
                                             cudaStream_t);                                      \
  template cudaError_t launch_cg_update<TV>(long long, int, double*, double*, const double*,     \
                                            const double*, TV*, double*, unsigned*, CgScalars*,  \
                                            double, int, cudaStream_t);                          \
  template cudaError_t launch_cg_direction<TV>(long long, int, const double*, const TV*,         \
                                               double*, TV*, int, double*, unsigned*,            \
                                               CgScalars*, cudaStream_t, double*);
TOPO_INST(double)
TOPO_INST(float)
#undef TOPO_INST

cudaError_t launch_check_conversions(const double* d, const float* f, long long n,
                                     unsigned long long* bad, cudaStream_t st) {
  topo::launch(k_check_conversions, dim3(kRedBlocks), kThreads, 0, st, d, f, n, bad);
  return cudaGetLastError();
}

}  // namespace topo
