// Kernels of the primal-dual interior-point method (Sec. 2-3) and of the OC methods (Sec. 4).
//
// IP.  With B(u) = (K_1 u, ..., K_m u), column e of B is L_e^T g_e with g_e = K0 u_e, and
// D = X^{-1} Phi + (xbar - X)^{-1} Psi is diagonal, so the augmented matrix of Eq. (nwtr2Z),
//   Z = [K(x) 0; 0 0] + [B; e^T] D^{-1} [B^T e],
// acts element by element:  s_e = (g_e^T v_e + v_lambda) / D_e,
//   (Z v)_u = K(x) v_u + sum_e L_e^T g_e s_e,   (Z v)_lambda = sum_e s_e.
// The right-hand side Eq. (nwtr2rhs) is Res1 + sum_e L_e^T g_e t_e, Res2 + sum_e t_e with
// t_e = tilde Res3_e / D_e.  The direction is completed element-wise: d_x from row 3 of
// Eq. (nwtr) and d_phi, d_psi from Eq. (phipsi1)-(phipsi2); the step is the 0.9 fraction-to-
// boundary rule of Sec. 3.3.  Row 3 of Eq. (nwt) uses the right-hand side
// F3 = -1/2 u^T K_i u - lambda - phi_i + psi_i (the printed matrix with the sign that makes the
// direction a Newton step of the KKT map).
//
// SIMP (Sec. 9).  hat B(u) = B(u) diag(c) W with c = p x~^(p-1) and the column-normalised density
// filter W (so e^T W = e^T).  The augmented Z is then the matrix above with columns c_e g_e and with
// D^{-1} replaced by M = W D^{-1} W^T: s = M (hat G^T v_u + e v_lambda), computed as one element pass,
// a filtered pass with the lambda-row reduction, and a second filter pass.  The filter is a stencil
// gather over the element grid (|o|_1 <= ceil(rmin) - 1) in a fixed order.
//
// OC.  The bisection on lambda of Algorithm OC compares sum_i x_i^NEW(lambda) with V using a
// double-double (error-free TwoSum) reduction rounded once at the end, so the decision does not
// depend on the summation order.
//
// All reductions write one partial per block; the last block to finish combines them in block
// order and updates the device-resident scalars.
#include "pairs.cuh"
#include "topo_internal.cuh"

namespace topo {

namespace {

__device__ __forceinline__ int loc_ox(int a) { return ((a & 3) == 1 || (a & 3) == 2) ? 1 : 0; }
__device__ __forceinline__ int loc_oy(int a) { return ((a & 3) >= 2) ? 1 : 0; }
__device__ __forceinline__ int loc_oz(int a) { return a >> 2; }
__device__ __forceinline__ int loc_of(int lx, int ly, int lz) {
  return (ly ? (lx ? 2 : 3) : (lx ? 1 : 0)) + 4 * lz;
}

template <int DIM>
__device__ __forceinline__ long long elem_node(const Dims& d, long long e, int a) {
  const int ex = (int)(e % d.nx), ey = (int)((e / d.nx) % d.ny);
  const int ez = (DIM == 3) ? (int)(e / ((long long)d.nx * d.ny)) : 0;
  return (ex + loc_ox(a)) + (long long)(d.nx + 1) * ((ey + loc_oy(a)) + (long long)(d.ny + 1) *
                                                                              (ez + loc_oz(a)));
}

// Block reduction of NV doubles; result valid in thread 0.
template <int NV>
__device__ void block_reduce(double (&v)[NV], int op_min) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double a = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double b = __shfl_down_sync(0xffffffffu, a, o);
      a = op_min ? fmin(a, b) : a + b;
    }
    v[q] = a;
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][wid] = v[q];
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double a = lane < nw ? sh[q][lane] : (op_min ? INFINITY : 0.0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double b = __shfl_down_sync(0xffffffffu, a, o);
        a = op_min ? fmin(a, b) : a + b;
      }
      v[q] = a;
    }
  }
}

// Writes the block's NV partials; returns true in the last block, with the combined values in
// tot (every thread of that block).
template <int NV>
__device__ bool last_block(double (&part)[NV], int op_min, double* partials, unsigned* counter,
                           double (&tot)[NV]) {
  __shared__ bool last;
  __shared__ double res[NV];
  block_reduce<NV>(part, op_min);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[(long long)q * gridDim.x + blockIdx.x] = part[q];
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    acc[q] = op_min ? INFINITY : 0.0;
    for (unsigned t = threadIdx.x; t < gridDim.x; t += blockDim.x) {
      const double b = __ldcg(partials + (long long)q * gridDim.x + t);
      acc[q] = op_min ? fmin(acc[q], b) : acc[q] + b;
    }
  }
  block_reduce<NV>(acc, op_min);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) res[q] = acc[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) tot[q] = res[q];
  if (threadIdx.x == 0) *counter = 0;
  return true;
}

// ---- Z operator ---------------------------------------------------------------------------
// s_e = (g_e^T v_e + v_lambda) Dinv_e and the lambda row (Z v)_lambda = sum_e s_e, written into
// y[n] according to MODE (0: Zv, 1: b - Zv, 2: Jacobi, 3: first Jacobi sweep).
template <int DIM, typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_z_elem(Dims d, const T* __restrict__ g,
                                                     const T* __restrict__ Dinv,
                                                     const T* __restrict__ v,
                                                     const T* __restrict__ b, T* __restrict__ y,
                                                     T* __restrict__ se, const double* zll,
                                                     double omega, double* partials,
                                                     unsigned* counter, const CgScalars* sc,
                                                     const double* wdev) {
  pdl_prologue();
  constexpr int NN = DIM == 2 ? 4 : 8, NE = NN * DIM;
  if (sc && sc[0].done) return;
  const long long m = d.elems();
  const long long n = d.dofs();
  const T vl = v[n];
  double part[1] = {0.0};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (long long)gridDim.x * blockDim.x) {
    T acc = vl;
#pragma unroll
    for (int a = 0; a < NN; ++a) {
      const long long nid = elem_node<DIM>(d, e, a);
#pragma unroll
      for (int c = 0; c < DIM; ++c) acc = fma(g[e * NE + a * DIM + c], v[DIM * nid + c], acc);
    }
    const T s = acc * Dinv[e];
    se[e] = s;
    part[0] += (double)s;
  }
  double tot[1];
  if (!last_block<1>(part, 0, partials, counter, tot)) return;
  if (threadIdx.x == 0) {
    const double q = tot[0];
    const double om = wdev ? *wdev : omega;
    double out;
    if (MODE == 0) out = q;
    else if (MODE == 1) out = (double)b[n] - q;
    else out = (double)v[n] + om * ((double)b[n] - q) / *zll;
    y[n] = (T)out;
  }
}

// (Z v)_u on the finest level: node gather of x_e K0 v_e + g_e s_e; MODE as k_z_elem.  MODE 3 also
// writes the lambda entry omega b_lambda / Z_ll.
template <int DIM, typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_z_node(Dims d, const T* __restrict__ K0,
                                                     const T* __restrict__ x,
                                                     const T* __restrict__ g,
                                                     const T* __restrict__ se,
                                                     const T* __restrict__ v,
                                                     const T* __restrict__ b, T* __restrict__ y,
                                                     const T* __restrict__ invd, T omega,
                                                     const uint8_t* __restrict__ fixed,
                                                     const double* zll, const CgScalars* sc,
                                                     const double* wdev) {
  pdl_prologue();
  constexpr int NN = DIM == 2 ? 4 : 8, NE = NN * DIM;
  if (sc && sc[0].done) return;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nodes = d.nodes();
  const long long n = nodes * DIM;
  if (MODE == 3 && node == 0)
    y[n] = (T)((wdev ? *wdev : (double)omega) * (double)b[n] / *zll);
  if (node >= nodes) return;
  const int nnx = d.nx + 1, nny = d.ny + 1;
  const int i = (int)(node % nnx), j = (int)((node / nnx) % nny);
  const int k = (DIM == 3) ? (int)(node / ((long long)nnx * nny)) : 0;
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
  if (MODE != 3) {
    for (int s = 0; s < NN; ++s) {
      const int dx = s & 1, dy = (s >> 1) & 1, dz = (DIM == 3) ? (s >> 2) : 0;
      const int ex = i - 1 + dx, ey = j - 1 + dy, ez = (DIM == 3) ? k - 1 + dz : 0;
      if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny) continue;
      if (DIM == 3 && (ez < 0 || ez >= d.nz)) continue;
      const int loc = loc_of(1 - dx, 1 - dy, DIM == 3 ? 1 - dz : 0);
      const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
      T ve[NE];
#pragma unroll
      for (int a = 0; a < NN; ++a) {
        const long long nid = elem_node<DIM>(d, e, a);
#pragma unroll
        for (int c = 0; c < DIM; ++c) ve[a * DIM + c] = v[DIM * nid + c];
      }
      const T xe = x[e], s_e = se[e];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const T* row = K0 + (loc * DIM + c) * NE;
        T t = T(0);
#pragma unroll
        for (int q = 0; q < NE; ++q) t = fma(row[q], ve[q], t);
        acc[c] = fma(xe, t, acc[c]);
        acc[c] = fma(g[e * NE + loc * DIM + c], s_e, acc[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const long long id = DIM * node + c;
    T out;
    if (fixed[id]) out = T(0);
    else if (MODE == 0) out = acc[c];
    else if (MODE == 1) out = b[id] - acc[c];
    else if (MODE == 2) out = v[id] + omega * invd[id] * (b[id] - acc[c]);
    else out = omega * invd[id] * b[id];
    y[id] = out;
  }
}

// (Z v)_u on the finest level in float pairs, for mixed-precision IP systems: k_z_node's MODE 0
// with K0 staged in shared memory as pairs and x, g, s_e and v converted from FP64 as they load.
// The FP64 pipe of this GPU runs at a sixtieth of the FP32 rate, and the node pass is 80 FP64
// multiply-adds per node.  The result hi + lo goes to FP64 (about 48 significant bits, as the
// K systems' pair operator).
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_z_node_df(Dims d, const double* __restrict__ K0,
                                                        const double* __restrict__ x,
                                                        const double* __restrict__ g,
                                                        const double* __restrict__ se,
                                                        const double* __restrict__ v,
                                                        double* __restrict__ y,
                                                        const uint8_t* __restrict__ fixed,
                                                        const CgScalars* sc) {
  pdl_prologue();
  constexpr int NN = DIM == 2 ? 4 : 8, NE = NN * DIM;
  __shared__ f2 k0s[NE * NE];
  if (sc && sc[0].done) return;  // the same for the whole block
  for (int t = threadIdx.x; t < NE * NE; t += blockDim.x) k0s[t] = df_from_double(K0[t]);
  __syncthreads();
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nodes = d.nodes();
  if (node >= nodes) return;
  const int nnx = d.nx + 1, nny = d.ny + 1;
  const int i = (int)(node % nnx), j = (int)((node / nnx) % nny);
  const int k = (DIM == 3) ? (int)(node / ((long long)nnx * nny)) : 0;
  PairNum acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = PairNum{{0.0f, 0.0f}};
  for (int s = 0; s < NN; ++s) {
    const int dx = s & 1, dy = (s >> 1) & 1, dz = (DIM == 3) ? (s >> 2) : 0;
    const int ex = i - 1 + dx, ey = j - 1 + dy, ez = (DIM == 3) ? k - 1 + dz : 0;
    if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny) continue;
    if (DIM == 3 && (ez < 0 || ez >= d.nz)) continue;
    const int loc = loc_of(1 - dx, 1 - dy, DIM == 3 ? 1 - dz : 0);
    const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
    PairNum ve[NE];
#pragma unroll
    for (int a = 0; a < NN; ++a) {
      const long long nid = elem_node<DIM>(d, e, a);
#pragma unroll
      for (int c = 0; c < DIM; ++c) ve[a * DIM + c] = PairNum{df_from_double(v[DIM * nid + c])};
    }
    const PairNum xe{df_from_double(x[e])}, s_e{df_from_double(se[e])};
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const f2* row = k0s + (loc * DIM + c) * NE;
      PairNum t{{0.0f, 0.0f}};
#pragma unroll
      for (int q = 0; q < NE; ++q) t = fma(PairNum{row[q]}, ve[q], t);
      acc[c] = fma(xe, t, acc[c]);
      acc[c] = fma(PairNum{df_from_double(g[e * NE + loc * DIM + c])}, s_e, acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const long long id = DIM * node + c;
    y[id] = fixed[id] ? 0.0
                      : __dadd_rn(double_from_float(acc[c].v.h), double_from_float(acc[c].v.l));
  }
}

// ---- IP element and node kernels ---------------------------------------------------------
// Per element at z = (u, lambda, x, phi, psi) and barrier (s, r):
//   g_e = K0 u_e, F3 = -1/2 u_e^T g_e - lambda - phi + psi, Res4 = s - phi x,
//   Res5 = r - psi (xbar - x), tR3 = F3 - Res4/x + Res5/(xbar - x), D = phi/x + psi/(xbar - x),
//   Dinv = 1/D, t = tR3 Dinv.  Sums: sum x, sum t, ||tR3||^2, ||phi||^2, ||psi||^2, sum Dinv.
// e3 != null (SIMP, Sec. 9): F3 takes the filtered energy term -e3_e in place of -1/2 u_e^T g_e.
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_ip_elem(Dims d, const double* __restrict__ K0,
                                                      const double* __restrict__ u,
                                                      const double* __restrict__ x,
                                                      const double* __restrict__ phi,
                                                      const double* __restrict__ psi,
                                                      IpScalars* ip, double* __restrict__ g,
                                                      double* __restrict__ tR3,
                                                      double* __restrict__ Dinv,
                                                      double* __restrict__ t, double* partials,
                                                      unsigned* counter,
                                                      const double* __restrict__ e3) {
  pdl_prologue();
  constexpr int NN = DIM == 2 ? 4 : 8, NE = NN * DIM;
  const long long m = d.elems();
  const double lam = ip->lam, s = ip->s, r = ip->r, xbar = ip->xbar;
  double part[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (long long)gridDim.x * blockDim.x) {
    double ue[NE];
#pragma unroll
    for (int a = 0; a < NN; ++a) {
      const long long nid = elem_node<DIM>(d, e, a);
#pragma unroll
      for (int c = 0; c < DIM; ++c) ue[a * DIM + c] = u[DIM * nid + c];
    }
    double en = 0.0;
    for (int q = 0; q < NE; ++q) {
      double acc = 0.0;
#pragma unroll
      for (int p = 0; p < NE; ++p) acc = fma(__ldg(K0 + q * NE + p), ue[p], acc);
      g[e * NE + q] = acc;
      en = fma(ue[q], acc, en);
    }
    const double xe = x[e], ph = phi[e], ps = psi[e];
    const double xu = xbar - xe;
    const double F3 = (e3 ? -e3[e] : -0.5 * en) - lam - ph + ps;
    const double R4 = s - ph * xe, R5 = r - ps * xu;
    const double tr = F3 - R4 / xe + R5 / xu;
    const double De = ph / xe + ps / xu;
    const double di = 1.0 / De;
    tR3[e] = tr;
    Dinv[e] = di;
    t[e] = tr * di;
    part[0] += xe;
    part[1] += tr * di;
    part[2] = fma(tr, tr, part[2]);
    part[3] = fma(ph, ph, part[3]);
    part[4] = fma(ps, ps, part[4]);
    part[5] += di;
    part[6] = fma(ph, xe, part[6]);  // the complementarity terms of the scaled KKT residual
    part[7] = fma(ps, xu, part[7]);
    part[8] = fma(xe, xe, part[8]);
    part[9] = fma(xu, xu, part[9]);
  }
  double tot[10];
  if (!last_block<10>(part, 0, partials, counter, tot)) return;
  if (threadIdx.x == 0) {
    ip->sum_x = tot[0];
    ip->sum_t = tot[1];
    ip->nrm_tr3 = sqrt(tot[2]);
    ip->nrm_phi = sqrt(tot[3]);
    ip->nrm_psi = sqrt(tot[4]);
    ip->zll = tot[5];
    ip->comp_phi = tot[6];
    ip->comp_psi = tot[7];
    ip->nrm_x = sqrt(tot[8]);
    ip->nrm_xu = sqrt(tot[9]);
  }
}

// Per node: Res1 = f - K(x) u; rhs_u = Res1 + sum_e g_e t_e; w = sum_e g_e Dinv_e (the Z_ul
// column); invd = 1 / (sum_e x_e K0_ii + g_e,i^2 Dinv_e); ||Res1||^2.  Last block: rhs_lambda.
// gk: the K0 u_e used for K(x) u (SIMP: the unscaled columns, while g holds c_e K0 u_e).
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_ip_node(Dims d, const double* __restrict__ K0,
                                                      const double* __restrict__ x,
                                                      const double* __restrict__ u,
                                                      const double* __restrict__ f,
                                                      const double* __restrict__ gk,
                                                      const double* __restrict__ g,
                                                      const double* __restrict__ t,
                                                      const double* __restrict__ Dinv,
                                                      const uint8_t* __restrict__ fixed,
                                                      double* __restrict__ rhs,
                                                      double* __restrict__ w,
                                                      double* __restrict__ invd, IpScalars* ip,
                                                      double* partials, unsigned* counter) {
  pdl_prologue();
  constexpr int NN = DIM == 2 ? 4 : 8, NE = NN * DIM;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nodes = d.nodes();
  double part[1] = {0.0};
  if (node < nodes) {
    const int nnx = d.nx + 1, nny = d.ny + 1;
    const int i = (int)(node % nnx), j = (int)((node / nnx) % nny);
    const int k = (DIM == 3) ? (int)(node / ((long long)nnx * nny)) : 0;
    double ku[DIM] = {}, gt[DIM] = {}, gw[DIM] = {}, dg[DIM] = {};
    for (int s = 0; s < NN; ++s) {
      const int dx = s & 1, dy = (s >> 1) & 1, dz = (DIM == 3) ? (s >> 2) : 0;
      const int ex = i - 1 + dx, ey = j - 1 + dy, ez = (DIM == 3) ? k - 1 + dz : 0;
      if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny) continue;
      if (DIM == 3 && (ez < 0 || ez >= d.nz)) continue;
      const int loc = loc_of(1 - dx, 1 - dy, DIM == 3 ? 1 - dz : 0);
      const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
      const double xe = x[e], te = t[e], de = Dinv[e];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const double gi = g[e * NE + loc * DIM + c];
        // K(x) u row = x_e (K0 u_e)_row
        ku[c] = fma(xe, gk[e * NE + loc * DIM + c], ku[c]);
        gt[c] = fma(gi, te, gt[c]);
        gw[c] = fma(gi, de, gw[c]);
        dg[c] = fma(xe, K0[(loc * DIM + c) * NE + loc * DIM + c], dg[c]);
        dg[c] = fma(gi * gi, de, dg[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const long long id = DIM * node + c;
      if (fixed[id]) {
        rhs[id] = 0.0;
        w[id] = 0.0;
        invd[id] = 1.0;
      } else {
        const double r1 = f[id] - ku[c];
        rhs[id] = r1 + gt[c];
        w[id] = gw[c];
        invd[id] = dg[c] > 0.0 ? 1.0 / dg[c] : 1.0;
        part[0] = fma(r1, r1, part[0]);
      }
    }
  }
  double tot[1];
  if (!last_block<1>(part, 0, partials, counter, tot)) return;
  if (threadIdx.x == 0) {
    ip->nrm_res1 = sqrt(tot[0]);
    const double res2 = ip->V - ip->sum_x;
    ip->res2 = res2;
    rhs[d.dofs()] = res2 + ip->sum_t;
  }
}

// Direction completion and step length: d_x = (g_e^T d_u,e + d_lambda - tR3) Dinv,
// d_phi = (Res4 - phi d_x)/x, d_psi = (Res5 + psi d_x)/(xbar - x); minima of the ratios of the
// 0.9 rule over x (both bounds), phi and psi.  bt != null (SIMP): bt_e = (hat B^T d_u)_e replaces
// g_e^T d_u,e.
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_ip_recover(Dims d, const double* __restrict__ g,
                                                         const double* __restrict__ du,
                                                         const double* __restrict__ tR3,
                                                         const double* __restrict__ Dinv,
                                                         const double* __restrict__ x,
                                                         const double* __restrict__ phi,
                                                         const double* __restrict__ psi,
                                                         double* __restrict__ dx,
                                                         double* __restrict__ dphi,
                                                         double* __restrict__ dpsi,
                                                         IpScalars* ip, double* partials,
                                                         unsigned* counter,
                                                         const double* __restrict__ bt) {
  pdl_prologue();
  constexpr int NN = DIM == 2 ? 4 : 8, NE = NN * DIM;
  const long long m = d.elems();
  const long long n = d.dofs();
  const double dl = du[n];
  const double s = ip->s, r = ip->r, xbar = ip->xbar;
  double part[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (long long)gridDim.x * blockDim.x) {
    double acc = dl - tR3[e];
    if (bt) {
      acc += bt[e];
    } else {
#pragma unroll
      for (int a = 0; a < NN; ++a) {
        const long long nid = elem_node<DIM>(d, e, a);
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc = fma(g[e * NE + a * DIM + c], du[DIM * nid + c], acc);
      }
    }
    const double ddx = acc * Dinv[e];
    const double xe = x[e], ph = phi[e], ps = psi[e], xu = xbar - xe;
    const double R4 = s - ph * xe, R5 = r - ps * xu;
    const double dph = (R4 - ph * ddx) / xe;
    const double dps = (R5 + ps * ddx) / xu;
    dx[e] = ddx;
    dphi[e] = dph;
    dpsi[e] = dps;
    if (ddx < 0.0) part[0] = fmin(part[0], -xe / ddx);
    if (ddx > 0.0) part[1] = fmin(part[1], xu / ddx);
    if (dph < 0.0) part[2] = fmin(part[2], -ph / dph);
    if (dps < 0.0) part[3] = fmin(part[3], -ps / dps);
  }
  double tot[4];
  if (!last_block<4>(part, 1, partials, counter, tot)) return;
  if (threadIdx.x == 0) {
    const double fr = ip->frac;
    double a = fmin(1.0, fmin(fr * tot[0], fr * tot[1]));
    if (ip->step_all) a = fmin(a, fmin(fr * tot[2], fr * tot[3]));
    ip->alpha = a;
    ip->dlam = dl;
  }
}

// z += alpha d on the element variables and lambda.
__global__ void k_ip_update_elem(long long m, double* x, double* phi, double* psi,
                                 const double* dx, const double* dphi, const double* dpsi,
                                 IpScalars* ip) {
  pdl_prologue();
  const double a = ip->alpha;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) ip->lam += a * ip->dlam;
  if (e >= m) return;
  x[e] = fma(a, dx[e], x[e]);
  phi[e] = fma(a, dphi[e], phi[e]);
  psi[e] = fma(a, dpsi[e], psi[e]);
}

__global__ void k_axpy_alpha(long long n, double* u, const double* du, const IpScalars* ip) {
  pdl_prologue();
  const double a = ip->alpha;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    u[i] = fma(a, du[i], u[i]);
}

// ---- SIMP density filter (Sec. 9) ---------------------------------------------------------
// The stencil of element (ex, ey, ez): in-grid offsets o with |o|_1 <= R, weight hat W = rmin -
// |o|_1 (> 0 since R = ceil(rmin) - 1 < rmin); hat W is symmetric, so row and column sums agree.
// Each sum runs over the offsets in a fixed order (z, y, x ascending): results do not depend on
// the launch.
template <int DIM>
__device__ __forceinline__ void elem_coords(const Dims& d, long long e, int& ex, int& ey, int& ez) {
  ex = (int)(e % d.nx);
  ey = (int)((e / d.nx) % d.ny);
  ez = (DIM == 3) ? (int)(e / ((long long)d.nx * d.ny)) : 0;
}

// sum over the stencil of w * a_j * b_j (a or b may be null = 1).
template <int DIM>
__device__ double stencil_sum(const Dims& d, long long e, double rmin, int R,
                              const double* __restrict__ a, const double* __restrict__ b) {
  int ex, ey, ez;
  elem_coords<DIM>(d, e, ex, ey, ez);
  const int zr = DIM == 3 ? R : 0;
  double acc = 0.0;
  for (int dz = -zr; dz <= zr; ++dz) {
    const int jz = ez + dz;
    if (DIM == 3 && (jz < 0 || jz >= d.nz)) continue;
    const int rz = R - abs(dz);
    for (int dy = -rz; dy <= rz; ++dy) {
      const int jy = ey + dy;
      if (jy < 0 || jy >= d.ny) continue;
      const int ry = rz - abs(dy);
      for (int dx = -ry; dx <= ry; ++dx) {
        const int jx = ex + dx;
        if (jx < 0 || jx >= d.nx) continue;
        const double w = rmin - (double)(abs(dx) + abs(dy) + abs(dz));
        const long long j = jx + (long long)d.nx * (jy + (long long)d.ny * jz);
        const double v = a ? (b ? a[j] * b[j] : a[j]) : (b ? b[j] : 1.0);
        acc = fma(w, v, acc);
      }
    }
  }
  return acc;
}

template <int DIM>
__global__ void k_filter_colsum(Dims d, double rmin, int R, double* __restrict__ invS) {
  pdl_prologue();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.elems()) return;
  invS[e] = 1.0 / stencil_sum<DIM>(d, e, rmin, R, nullptr, nullptr);
}

// x~ = W x (x~_k = sum_i hat W_ki x_i / S_i), rho = x~^p, c = p x~^(p-1).
template <int DIM>
__global__ void k_simp_density(Dims d, double rmin, int R, const double* __restrict__ invS,
                               const double* __restrict__ x, double p, double* __restrict__ xt,
                               double* __restrict__ rho, double* __restrict__ c) {
  pdl_prologue();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.elems()) return;
  const double v = stencil_sum<DIM>(d, e, rmin, R, x, invS);
  xt[e] = v;
  rho[e] = p == 1.0 ? v : pow(v, p);
  c[e] = p == 1.0 ? 1.0 : p * pow(v, p - 1.0);
}

// out_i = post (W^T (pre a))_i = post / S_i sum_k hat W_ik pre_k a_k  (pre may be null = 1).
template <int DIM>
__global__ void k_filter_t(Dims d, double rmin, int R, const double* __restrict__ invS,
                           const double* __restrict__ a, const double* __restrict__ pre,
                           double post, double* __restrict__ out, const CgScalars* sc) {
  pdl_prologue();
  if (sc && sc[0].done) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.elems()) return;
  out[e] = post * invS[e] * stencil_sum<DIM>(d, e, rmin, R, a, pre);
}

// out_k = (W a)_k = sum_j hat W_kj a_j / S_j.
template <int DIM>
__global__ void k_filter_w(Dims d, double rmin, int R, const double* __restrict__ invS,
                           const double* __restrict__ a, double* __restrict__ out,
                           const CgScalars* sc) {
  pdl_prologue();
  if (sc && sc[0].done) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.elems()) return;
  out[e] = stencil_sum<DIM>(d, e, rmin, R, a, invS);
}

// Between the element and node passes of the SIMP residuals: th = W t (the right-hand side's
// element weights), Dm = W Dinv = (W D^{-1} W^T) e, the row sums of W D^{-1} W^T (every column of W
// sums to 1, so W^T e = e), and gh_e = c_e g_e.  The hierarchy's element-local Z keeps
// diag(Dm) in place of W D^{-1} W^T: exact on the lambda row and column and on constant element
// fields, and above Z in the Loewner order (diag(Dm) - W D^{-1} W^T is a weighted graph
// Laplacian).
template <int DIM>
__global__ void k_simp_mid(Dims d, double rmin, int R, const double* __restrict__ invS,
                           const double* __restrict__ t, const double* __restrict__ Dinv,
                           const double* __restrict__ g, const double* __restrict__ c,
                           double* __restrict__ th, double* __restrict__ Dm,
                           double* __restrict__ gh) {
  pdl_prologue();
  constexpr int NE = (DIM == 2 ? 4 : 8) * DIM;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.elems()) return;
  th[e] = stencil_sum<DIM>(d, e, rmin, R, t, invS);
  Dm[e] = stencil_sum<DIM>(d, e, rmin, R, Dinv, invS);
  const double ce = c[e];
#pragma unroll
  for (int q = 0; q < NE; ++q) gh[e * NE + q] = ce * g[e * NE + q];
}

// a_e = g_e^T v_e.
template <int DIM>
__global__ void k_elem_gdot(Dims d, const double* __restrict__ g, const double* __restrict__ v,
                            double* __restrict__ a, const CgScalars* sc) {
  pdl_prologue();
  constexpr int NN = DIM == 2 ? 4 : 8, NE = NN * DIM;
  if (sc && sc[0].done) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.elems()) return;
  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < NN; ++q) {
    const long long nid = elem_node<DIM>(d, e, q);
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc = fma(g[e * NE + q * DIM + c], v[DIM * nid + c], acc);
  }
  a[e] = acc;
}

// sb_i = Dinv_i ((W^T a)_i + v_lambda) and the lambda row y_lambda = sum_i sb_i
// (= e^T W sb, since every column of W sums to 1).
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_simp_zt(Dims d, double rmin, int R,
                                                      const double* __restrict__ invS,
                                                      const double* __restrict__ a,
                                                      const double* __restrict__ Dinv,
                                                      const double* __restrict__ v,
                                                      double* __restrict__ y,
                                                      double* __restrict__ sb, double* partials,
                                                      unsigned* counter, const CgScalars* sc) {
  pdl_prologue();
  if (sc && sc[0].done) return;
  const long long m = d.elems();
  const double vl = v[d.dofs()];
  double part[1] = {0.0};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (long long)gridDim.x * blockDim.x) {
    const double s = Dinv[e] * fma(invS[e], stencil_sum<DIM>(d, e, rmin, R, a, nullptr), vl);
    sb[e] = s;
    part[0] += s;
  }
  double tot[1];
  if (!last_block<1>(part, 0, partials, counter, tot)) return;
  if (threadIdx.x == 0) y[d.dofs()] = tot[0];
}

// ---- OC kernels --------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void dd_add(double& hi, double& lo, double bh, double bl) {
  double s, e;
  two_sum(hi, bh, s, e);
  e += lo + bl;
  two_sum(s, e, hi, lo);
}

__device__ __forceinline__ double oc_new(double xo, double E, double lam, double xlow,
                                         double xbar) {
  return fmin(fmax(xo * E / lam, xlow), xbar);
}

// One bisection step of Algorithm OC: x^NEW(lambda_mid), its sum in double-double, and in the
// last block: "sum > V" raises the lower end, otherwise lowers the upper end; next midpoint.
__global__ void __launch_bounds__(kThreads) k_oc_bisect(long long m, const double* __restrict__ x,
                                                        const double* __restrict__ E,
                                                        OcScalars* oc, double* partials,
                                                        unsigned* counter) {
  pdl_prologue();
  if (oc->hi - oc->lo <= oc->tau) return;
  const double lam = 0.5 * (oc->hi + oc->lo);
  const double xlow = oc->xlow, xbar = oc->xbar;
  double hi = 0.0, lo = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (long long)gridDim.x * blockDim.x)
    dd_add(hi, lo, oc_new(x[e], E[e], lam, xlow, xbar), 0.0);
  // warp and block combination of (hi, lo) pairs in a fixed order
  __shared__ double sh[2][32];
  __shared__ bool last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double bh = __shfl_down_sync(0xffffffffu, hi, o);
    const double bl = __shfl_down_sync(0xffffffffu, lo, o);
    dd_add(hi, lo, bh, bl);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = hi;
    sh[1][wid] = lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double h = 0.0, l = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) dd_add(h, l, sh[0][w], sh[1][w]);
    partials[2 * blockIdx.x] = h;
    partials[2 * blockIdx.x + 1] = l;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  // the last block combines the blocks' pairs: thread t takes blocks t, t + blockDim, ... in order,
  // then the warp and block combinations above, in a fixed order (one thread walking all the
  // blocks' pairs from L2 took about 0.25 ms per step)
  double h = 0.0, l = 0.0;
  for (unsigned bidx = threadIdx.x; bidx < gridDim.x; bidx += blockDim.x)
    dd_add(h, l, __ldcg(partials + 2 * bidx), __ldcg(partials + 2 * bidx + 1));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double bh = __shfl_down_sync(0xffffffffu, h, o);
    const double bl = __shfl_down_sync(0xffffffffu, l, o);
    dd_add(h, l, bh, bl);
  }
  __syncthreads();  // (sh is reused)
  if (lane == 0) {
    sh[0][wid] = h;
    sh[1][wid] = l;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  h = 0.0;
  l = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) dd_add(h, l, sh[0][w], sh[1][w]);
  const double total = h + l;  // round the double-double once
  if (total > oc->V) oc->lo = lam;
  else oc->hi = lam;
  oc->lam_last = lam;
  oc->steps += 1;
  *counter = 0;
}

// x_out = x^NEW(lambda_last); optionally averaged with x_avg (AOC: 1/2 (x1 + x2)).
__global__ void k_oc_apply(long long m, const double* __restrict__ x, const double* __restrict__ E,
                           const OcScalars* oc, double* __restrict__ xout) {
  pdl_prologue();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  xout[e] = oc_new(x[e], E[e], oc->lam_last, oc->xlow, oc->xbar);
}

__global__ void k_pow(long long m, double* E, double q) {
  pdl_prologue();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) E[e] = pow(fmax(E[e], 0.0), q);
}

__global__ void k_average(long long m, const double* a, const double* b, double* out) {
  pdl_prologue();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) out[e] = 0.5 * (a[e] + b[e]);
}

inline unsigned red_grid(long long n) {
  const long long b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b < kRedBlocks ? (b < 1 ? 1 : b) : kRedBlocks);
}

}  // namespace

template <typename T>
cudaError_t launch_z_apply_fine(const Dims& d, int mode, const T* K0, const T* x, const T* g,
                                const T* Dinv, T* se, const T* v, const T* b, T* y, const T* invd,
                                T omega, const uint8_t* fixed, const double* zll, double* partials,
                                unsigned* counter, const CgScalars* sc, cudaStream_t st,
                                const double* wdev) {
  const unsigned ge = red_grid(d.elems());
  const unsigned gn = blocks_for(d.nodes());
#define TOPO_ZF(DIM, MODE)                                                                      \
  do {                                                                                          \
    if (MODE != 3)                                                                              \
      topo::launch(k_z_elem<DIM, T, MODE>, ge, kThreads, 0, st, d, g, Dinv, v, b, y, se, zll, omega,      \
                                                      partials, counter, sc, wdev);             \
    topo::launch(k_z_node<DIM, T, MODE>, gn, kThreads, 0, st, d, K0, x, g, se, v, b, y, invd, omega,      \
                                                    fixed, zll, sc, wdev);                      \
  } while (0)
  if (d.dim == 2) {
    switch (mode) {
      case 0: TOPO_ZF(2, 0); break;
      case 1: TOPO_ZF(2, 1); break;
      case 2: TOPO_ZF(2, 2); break;
      default: TOPO_ZF(2, 3);
    }
  } else {
    switch (mode) {
      case 0: TOPO_ZF(3, 0); break;
      case 1: TOPO_ZF(3, 1); break;
      case 2: TOPO_ZF(3, 2); break;
      default: TOPO_ZF(3, 3);
    }
  }
#undef TOPO_ZF
  return cudaGetLastError();
}
template cudaError_t launch_z_apply_fine<double>(const Dims&, int, const double*, const double*,
                                                 const double*, const double*, double*,
                                                 const double*, const double*, double*,
                                                 const double*, double, const uint8_t*,
                                                 const double*, double*, unsigned*,
                                                 const CgScalars*, cudaStream_t, const double*);
template cudaError_t launch_z_apply_fine<float>(const Dims&, int, const float*, const float*,
                                                const float*, const float*, float*, const float*,
                                                const float*, float*, const float*, float,
                                                const uint8_t*, const double*, double*, unsigned*,
                                                const CgScalars*, cudaStream_t, const double*);


cudaError_t launch_z_apply_fine_df(const Dims& d, const double* K0, const double* x,
                                   const double* g, const double* Dinv, double* se,
                                   const double* v, double* y, const uint8_t* fixed,
                                   const double* zll, double* partials, unsigned* counter,
                                   const CgScalars* sc, cudaStream_t st) {
  const unsigned ge = red_grid(d.elems());
  const unsigned gn = blocks_for(d.nodes());
  if (d.dim == 2) {
    topo::launch(k_z_elem<2, double, 0>, ge, kThreads, 0, st, d, g, Dinv, v,
                 (const double*)nullptr, y, se, zll, 1.0, partials, counter, sc,
                 (const double*)nullptr);
    topo::launch(k_z_node_df<2>, gn, kThreads, 0, st, d, K0, x, g, (const double*)se, v, y, fixed,
                 sc);
  } else {
    topo::launch(k_z_elem<3, double, 0>, ge, kThreads, 0, st, d, g, Dinv, v,
                 (const double*)nullptr, y, se, zll, 1.0, partials, counter, sc,
                 (const double*)nullptr);
    topo::launch(k_z_node_df<3>, gn, kThreads, 0, st, d, K0, x, g, (const double*)se, v, y, fixed,
                 sc);
  }
  return cudaGetLastError();
}

cudaError_t launch_ip_residuals(const Dims& d, const double* K0, const double* u, const double* x,
                                const double* phi, const double* psi, const double* f,
                                const uint8_t* fixed, IpScalars* ip, double* g, double* tR3,
                                double* Dinv, double* t, double* rhs, double* w, double* invd,
                                double* partials, unsigned* counter, cudaStream_t st,
                                const SimpArgs* sa) {
  const unsigned ge = red_grid(d.elems());
  const unsigned gm = blocks_for(d.elems());
  const double* e3 = nullptr;
  if (sa) {  // x~, rho, c; E = u_e^T K0 u_e; e3 = 1/2 W^T (c E)
    cudaError_t e = launch_simp_density(d, *sa, x, st);
    if (e != cudaSuccess) return e;
    e = launch_element_energy(d, K0, u, u, sa->E, 1.0, st);
    if (e != cudaSuccess) return e;
    if (d.dim == 2)
      topo::launch(k_filter_t<2>, gm, kThreads, 0, st, d, sa->rmin, sa->R, sa->invS,
                   (const double*)sa->E, (const double*)sa->c, 0.5, sa->e3, (const CgScalars*)nullptr);
    else
      topo::launch(k_filter_t<3>, gm, kThreads, 0, st, d, sa->rmin, sa->R, sa->invS,
                   (const double*)sa->E, (const double*)sa->c, 0.5, sa->e3, (const CgScalars*)nullptr);
    e3 = sa->e3;
  }
  if (d.dim == 2)
    topo::launch(k_ip_elem<2>, ge, kThreads, 0, st, d, K0, u, x, phi, psi, ip, g, tR3, Dinv, t,
                 partials, counter, e3);
  else
    topo::launch(k_ip_elem<3>, ge, kThreads, 0, st, d, K0, u, x, phi, psi, ip, g, tR3, Dinv, t,
                 partials, counter, e3);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // node pass: K(x) u with the unscaled g; Z's right-hand side, column and diagonal with the
  // hierarchy's element data
  const double* xk = x;
  const double* gz = g;
  const double* tz = t;
  const double* dz = Dinv;
  if (sa) {
    if (d.dim == 2)
      topo::launch(k_simp_mid<2>, gm, kThreads, 0, st, d, sa->rmin, sa->R, sa->invS,
                   (const double*)t, (const double*)Dinv, (const double*)g, (const double*)sa->c,
                   sa->th, sa->Dm, sa->gh);
    else
      topo::launch(k_simp_mid<3>, gm, kThreads, 0, st, d, sa->rmin, sa->R, sa->invS,
                   (const double*)t, (const double*)Dinv, (const double*)g, (const double*)sa->c,
                   sa->th, sa->Dm, sa->gh);
    xk = sa->rho;
    gz = sa->gh;
    tz = sa->th;
    dz = sa->Dm;
  }
  const unsigned gn = blocks_for(d.nodes());
  if (d.dim == 2)
    topo::launch(k_ip_node<2>, gn, kThreads, 0, st, d, K0, xk, u, f, (const double*)g, gz, tz, dz,
                 fixed, rhs, w, invd, ip, partials, counter);
  else
    topo::launch(k_ip_node<3>, gn, kThreads, 0, st, d, K0, xk, u, f, (const double*)g, gz, tz, dz,
                 fixed, rhs, w, invd, ip, partials, counter);
  return cudaGetLastError();
}

cudaError_t launch_ip_recover_update(const Dims& d, const double* g, const double* du,
                                     const double* tR3, const double* Dinv, double* u, double* x,
                                     double* phi, double* psi, double* dx, double* dphi,
                                     double* dpsi, IpScalars* ip, double* partials,
                                     unsigned* counter, cudaStream_t st, const SimpArgs* sa) {
  const unsigned ge = red_grid(d.elems());
  const double* bt = nullptr;
  if (sa) {  // bt = hat B^T d_u = W^T (gh^T d_u)
    const unsigned gm = blocks_for(d.elems());
    if (d.dim == 2) {
      topo::launch(k_elem_gdot<2>, gm, kThreads, 0, st, d, (const double*)sa->gh, du, sa->ea,
                   (const CgScalars*)nullptr);
      topo::launch(k_filter_t<2>, gm, kThreads, 0, st, d, sa->rmin, sa->R, sa->invS,
                   (const double*)sa->ea, (const double*)nullptr, 1.0, sa->eb,
                   (const CgScalars*)nullptr);
    } else {
      topo::launch(k_elem_gdot<3>, gm, kThreads, 0, st, d, (const double*)sa->gh, du, sa->ea,
                   (const CgScalars*)nullptr);
      topo::launch(k_filter_t<3>, gm, kThreads, 0, st, d, sa->rmin, sa->R, sa->invS,
                   (const double*)sa->ea, (const double*)nullptr, 1.0, sa->eb,
                   (const CgScalars*)nullptr);
    }
    bt = sa->eb;
  }
  if (d.dim == 2)
    topo::launch(k_ip_recover<2>, ge, kThreads, 0, st, d, g, du, tR3, Dinv, x, phi, psi, dx, dphi,
                 dpsi, ip, partials, counter, bt);
  else
    topo::launch(k_ip_recover<3>, ge, kThreads, 0, st, d, g, du, tR3, Dinv, x, phi, psi, dx, dphi,
                 dpsi, ip, partials, counter, bt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long m = d.elems(), n = d.dofs();
  topo::launch(k_ip_update_elem, blocks_for(m), kThreads, 0, st, m, x, phi, psi, dx, dphi, dpsi, ip);
  topo::launch(k_axpy_alpha, red_grid(n), kThreads, 0, st, n, u, du, ip);
  return cudaGetLastError();
}

cudaError_t launch_filter_colsum(const Dims& d, double rmin, int R, double* invS,
                                 cudaStream_t st) {
  const long long m = d.elems();
  if (d.dim == 2)
    topo::launch(k_filter_colsum<2>, blocks_for(m), kThreads, 0, st, d, rmin, R, invS);
  else
    topo::launch(k_filter_colsum<3>, blocks_for(m), kThreads, 0, st, d, rmin, R, invS);
  return cudaGetLastError();
}

cudaError_t launch_simp_density(const Dims& d, const SimpArgs& sa, const double* x,
                                cudaStream_t st) {
  const unsigned gm = blocks_for(d.elems());
  if (d.dim == 2)
    topo::launch(k_simp_density<2>, gm, kThreads, 0, st, d, sa.rmin, sa.R, sa.invS, x, sa.p,
                 sa.xt, sa.rho, sa.c);
  else
    topo::launch(k_simp_density<3>, gm, kThreads, 0, st, d, sa.rmin, sa.R, sa.invS, x, sa.p,
                 sa.xt, sa.rho, sa.c);
  return cudaGetLastError();
}

cudaError_t launch_simp_z_apply(const Dims& d, const double* K0, const double* rho,
                                const double* gh, const double* Dinv, const double* invS,
                                double rmin, int R, double* ea, double* eb, double* se,
                                const double* v, double* y, const uint8_t* fixed,
                                double* partials, unsigned* counter, const CgScalars* sc,
                                cudaStream_t st, bool df) {
  const unsigned gm = blocks_for(d.elems());
  const unsigned ge = red_grid(d.elems());
  const unsigned gn = blocks_for(d.nodes());
#define TOPO_SZ(DIM)                                                                            \
  do {                                                                                          \
    topo::launch(k_elem_gdot<DIM>, gm, kThreads, 0, st, d, gh, v, ea, sc);                      \
    topo::launch(k_simp_zt<DIM>, ge, kThreads, 0, st, d, rmin, R, invS, (const double*)ea,      \
                 Dinv, v, y, eb, partials, counter, sc);                                        \
    topo::launch(k_filter_w<DIM>, gm, kThreads, 0, st, d, rmin, R, invS, (const double*)eb, se, \
                 sc);                                                                           \
    if (df)                                                                                     \
      topo::launch(k_z_node_df<DIM>, gn, kThreads, 0, st, d, K0, rho, gh, (const double*)se, v, \
                   y, fixed, sc);                                                               \
    else                                                                                        \
      topo::launch(k_z_node<DIM, double, 0>, gn, kThreads, 0, st, d, K0, rho, gh,               \
                   (const double*)se, v, (const double*)nullptr, y, (const double*)nullptr,     \
                   1.0, fixed, (const double*)nullptr, sc, (const double*)nullptr);             \
  } while (0)
  if (d.dim == 2)
    TOPO_SZ(2);
  else
    TOPO_SZ(3);
#undef TOPO_SZ
  return cudaGetLastError();
}

cudaError_t launch_oc_bisection(long long m, const double* x, const double* E, OcScalars* oc,
                                int steps, double* xout, double* partials, unsigned* counter,
                                cudaStream_t st) {
  const unsigned gr = red_grid(m);
  for (int k = 0; k < steps; ++k) {
    topo::launch(k_oc_bisect, gr, kThreads, 0, st, m, x, E, oc, partials, counter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  topo::launch(k_oc_apply, blocks_for(m), kThreads, 0, st, m, x, E, oc, xout);
  return cudaGetLastError();
}

cudaError_t launch_pow_inplace(long long m, double* E, double q, cudaStream_t st) {
  topo::launch(k_pow, blocks_for(m), kThreads, 0, st, m, E, q);
  return cudaGetLastError();
}

cudaError_t launch_average(long long m, const double* a, const double* b, double* out,
                           cudaStream_t st) {
  topo::launch(k_average, blocks_for(m), kThreads, 0, st, m, a, b, out);
  return cudaGetLastError();
}

}  // namespace topo
