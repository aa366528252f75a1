// Finest-level operator of the 3D trilinear hex grid in the element's Walsh-Hadamard basis
// (Eq. (to), Sec. 7): q = K(x) p with p^T q and alpha of Algorithm PCG.
//
// Element product.  For each displacement component the eight nodal values of an element are
// mapped to the coefficients of the modes (1, xi, eta, zeta, xi eta, eta zeta, xi zeta,
// xi eta zeta) by a three-stage Walsh-Hadamard butterfly (H, with H H^T = 8 I).  In that basis
// the cube element's stiffness Khat = T^-T K0 T^-1 has 45 nonzeros in five kinds of blocks:
//   normal strains (u_xi, v_eta, w_zeta): a on the diagonal, b off it;
//   the three shear pairs (u_eta, v_xi), (u_zeta, w_xi), (v_zeta, w_eta): s in every entry;
//   three bilinear pairs (u_xieta, w_etazeta), (u_xizeta, v_etazeta), (v_xieta, w_xizeta): p, q;
//   the triple (u_etazeta, v_xizeta, w_xieta): d on the diagonal, e off it;
//   the trilinear modes: h on the diagonal;
// and zero rows for the constant modes (rigid translations).  So K0 v_e costs two butterflies of
// 23 and 22 additions per component and about 43 scalings and additions: about 178 operations
// instead of 576 multiply-adds.  The host rebuilds T^T Khat T from the eight numbers and checks it
// against the quadrature K0 before enabling this path.
//
// Data movement.  One thread per element writes its 24 local forces to a buffer (entry-major, so
// that a warp writes contiguous memory); one thread per node then sums the contributions of its
// eight elements in a fixed order (deterministic, no atomics), masks fixed DOFs, and accumulates
// p^T q with the last-block finalisation of the other CG kernels.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "pairs.cuh"
#include "topo_internal.cuh"

namespace topo {

namespace {

__device__ __forceinline__ int hx_ox(int a) { return ((a & 3) == 1 || (a & 3) == 2) ? 1 : 0; }
__device__ __forceinline__ int hx_oy(int a) { return ((a & 3) >= 2) ? 1 : 0; }
__device__ __forceinline__ int hx_oz(int a) { return a >> 2; }

// Mode coefficients of one component: n[k][j][i] nodal values -> t = (xi, eta, zeta, xieta,
// etazeta, xizeta, xietazeta) (the constant mode is not needed).
template <typename T>
__device__ __forceinline__ void wht_fwd(const T n[2][2][2], T t[7]) {
  T Sx[2][2], Dx[2][2];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      Sx[k][j] = n[k][j][1] + n[k][j][0];
      Dx[k][j] = n[k][j][1] - n[k][j][0];
    }
  T SS[2], SD[2], DS[2], DD[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    SS[k] = Sx[k][1] + Sx[k][0];
    SD[k] = Sx[k][1] - Sx[k][0];
    DS[k] = Dx[k][1] + Dx[k][0];
    DD[k] = Dx[k][1] - Dx[k][0];
  }
  t[0] = DS[1] + DS[0];  // xi
  t[1] = SD[1] + SD[0];  // eta
  t[2] = SS[1] - SS[0];  // zeta
  t[3] = DD[1] + DD[0];  // xi eta
  t[4] = SD[1] - SD[0];  // eta zeta
  t[5] = DS[1] - DS[0];  // xi zeta
  t[6] = DD[1] - DD[0];  // xi eta zeta
}

// Nodal forces r[k][j][i] = sum_m H[m][node] g_m of one component (g of the constant mode = 0).
template <typename T>
__device__ __forceinline__ void wht_inv(const T g[7], T r[2][2][2]) {
  // z stage: A[mx][my][k]
  T A[2][2][2];
  A[0][0][0] = -g[2];
  A[0][0][1] = g[2];
  A[0][1][0] = g[1] - g[4];
  A[0][1][1] = g[1] + g[4];
  A[1][0][0] = g[0] - g[5];
  A[1][0][1] = g[0] + g[5];
  A[1][1][0] = g[3] - g[6];
  A[1][1][1] = g[3] + g[6];
  // y stage: B[mx][j][k]
  T B[2][2][2];
#pragma unroll
  for (int mx = 0; mx < 2; ++mx)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      B[mx][0][k] = A[mx][0][k] - A[mx][1][k];
      B[mx][1][k] = A[mx][0][k] + A[mx][1][k];
    }
  // x stage
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      r[k][j][0] = B[0][j][k] - B[1][j][k];
      r[k][j][1] = B[0][j][k] + B[1][j][k];
    }
}

template <typename T>
struct HexK {
  T a, b, s, p, q, d, e, h;
};

// Element forces of x_e K0 v_e: u, v, w mode coefficients in, forces out (in place).
template <typename T>
__device__ __forceinline__ void hex_khat(const HexK<T>& k, T xe, T tu[7], T tv[7], T tw[7]) {
  const T a = xe * k.a, b = xe * k.b, s = xe * k.s, p = xe * k.p, q = xe * k.q, d = xe * k.d,
          e = xe * k.e, h = xe * k.h;
  // normal strains
  const T S = tu[0] + tv[1] + tw[2];
  const T bS = b * S, ab = a - b;
  const T gux = fma(ab, tu[0], bS), gvy = fma(ab, tv[1], bS), gwz = fma(ab, tw[2], bS);
  // shears
  const T gxy = s * (tu[1] + tv[0]);
  const T gxz = s * (tu[2] + tw[0]);
  const T gyz = s * (tv[2] + tw[1]);
  // bilinear pairs
  const T guxy = fma(p, tu[3], q * tw[4]), gwyz = fma(q, tu[3], p * tw[4]);
  const T guxz = fma(p, tu[5], q * tv[4]), gvyz = fma(q, tu[5], p * tv[4]);
  const T gvxy = fma(p, tv[3], q * tw[5]), gwxz = fma(q, tv[3], p * tw[5]);
  // the triple
  const T Sd = tu[4] + tv[5] + tw[3];
  const T eS = e * Sd, de = d - e;
  const T guyz = fma(de, tu[4], eS), gvxz = fma(de, tv[5], eS), gwxy = fma(de, tw[3], eS);
  // trilinear
  const T guxyz = h * tu[6], gvxyz = h * tv[6], gwxyz = h * tw[6];
  tu[0] = gux; tu[1] = gxy; tu[2] = gxz; tu[3] = guxy; tu[4] = guyz; tu[5] = guxz; tu[6] = guxyz;
  tv[0] = gxy; tv[1] = gvy; tv[2] = gyz; tv[3] = gvxy; tv[4] = gvyz; tv[5] = gvxz; tv[6] = gvxyz;
  tw[0] = gxz; tw[1] = gyz; tw[2] = gwz; tw[3] = gwxy; tw[4] = gwyz; tw[5] = gwxz; tw[6] = gwxyz;
}

// One thread per element: R[(a * 3 + c) * m + e] = (x_e K0 v_e)_{a,c}.
__global__ void __launch_bounds__(kThreads) k_hex_elem(Dims d, HexK<double> k,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ v,
                                                       double* __restrict__ R,
                                                       const CgScalars* __restrict__ sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const long long m = d.elems();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const long long n = d.dofs();
  v += rhs * n;
  R += rhs * 24 * m;
  int ex, ey, ez;
  node_coords(e, d.nx, d.ny, 3, ex, ey, ez);
  const int nnx = d.nx + 1, nny = d.ny + 1;
  double nu[2][2][2], nv[2][2][2], nw[2][2][2];
#pragma unroll
  for (int kk = 0; kk < 2; ++kk)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const long long nid =
            TOPO_IDX((ex + i) + (long long)nnx * ((ey + j) + (long long)nny * (ez + kk)), d.nodes());
        nu[kk][j][i] = __ldg(v + 3 * nid);
        nv[kk][j][i] = __ldg(v + 3 * nid + 1);
        nw[kk][j][i] = __ldg(v + 3 * nid + 2);
      }
  double tu[7], tv[7], tw[7];
  wht_fwd(nu, tu);
  wht_fwd(nv, tv);
  wht_fwd(nw, tw);
  hex_khat(k, __ldg(x + e), tu, tv, tw);
  wht_inv(tu, nu);
  wht_inv(tv, nv);
  wht_inv(tw, nw);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int i = hx_ox(a), j = hx_oy(a), kk = hx_oz(a);
    R[(long long)(a * 3 + 0) * m + e] = nu[kk][j][i];
    R[(long long)(a * 3 + 1) * m + e] = nv[kk][j][i];
    R[(long long)(a * 3 + 2) * m + e] = nw[kk][j][i];
  }
}

// Block sum of one double per thread (deterministic tree), result valid in thread 0.
__device__ __forceinline__ double block_sum_hex(double v) {
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

// One thread per node: q = sum of the node's element forces (elements in the fixed order of
// node_apply), masked; p^T q and alpha = r^T y / p^T q by the last block.
__global__ void __launch_bounds__(kThreads) k_hex_gather_dot(Dims d, const double* __restrict__ R,
                                                             const double* __restrict__ p,
                                                             double* __restrict__ q,
                                                             const uint8_t* __restrict__ fixed,
                                                             double* partials, unsigned* counters,
                                                             CgScalars* sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc[rhs].done) return;
  const long long m = d.elems();
  const long long nodes = d.nodes();
  const long long n = nodes * 3;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  p += rhs * n;
  q += rhs * n;
  R += rhs * 24 * m;
  double part = 0.0;
  if (node < nodes) {
    int i, j, kk;
    node_coords(node, d.nx + 1, d.ny + 1, 3, i, j, kk);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int s = 0; s < 8; ++s) {
      const int dx = s & 1, dy = (s >> 1) & 1, dz = s >> 2;
      const int ex = i - 1 + dx, ey = j - 1 + dy, ez = kk - 1 + dz;
      if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny || ez < 0 || ez >= d.nz) continue;
      const int lx = 1 - dx, ly = 1 - dy, lz = 1 - dz;
      const int loc = (ly ? (lx ? 2 : 3) : (lx ? 1 : 0)) + 4 * lz;
      const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
      if (!TOPO_IN(e, m)) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] += __ldg(R + (long long)(loc * 3 + c) * m + e);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long id = 3 * node + c;
      if (!TOPO_IN(id, n)) continue;
      const double out = fixed[id] ? 0.0 : acc[c];
      q[id] = out;
      part = fma(p[id], out, part);
    }
  }
  const double bs = block_sum_hex(part);
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
  s = block_sum_hex(s);
  if (threadIdx.x == 0) {
    CgScalars& S = sc[rhs];
    S.pq = s;
    const double alpha = S.ry / s;
    if (!(s > 0.0) || !isfinite(alpha)) {
      S.status = TOPO_E_BREAKDOWN;
      S.done = 1;
      S.alpha = 0.0;
    } else {
      S.alpha = alpha;
    }
    counters[rhs] = 0;
  }
}

// ---- The same operator in pair-of-FP32 arithmetic (the mixed solver's outer operator) -------
// FP64 runs at about 2 operations per clock per SM on this part, so k_hex_elem is FP64-bound at
// ~178 operations per element.  Here every value is a float pair (about 48 bits): the three
// butterflies and the Khat blocks are the templates above on PairNum, p is split with integer
// operations, the element forces are stored as pairs (8 bytes, as the FP64 ones), the node sums
// run in pairs and q is rebuilt in FP64 with one add per DOF; p^T q is accumulated in pairs.
__global__ void __launch_bounds__(kThreads) k_hex_elem_df(Dims d, HexK<PairNum> k,
                                                          const float2* __restrict__ xdf,
                                                          const double* __restrict__ v,
                                                          float2* __restrict__ R,
                                                          const CgScalars* __restrict__ sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const long long m = d.elems();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const long long n = d.dofs();
  v += rhs * n;
  R += rhs * 24 * m;
  int ex, ey, ez;
  node_coords(e, d.nx, d.ny, 3, ex, ey, ez);
  const int nnx = d.nx + 1, nny = d.ny + 1;
  PairNum nu[2][2][2], nv[2][2][2], nw[2][2][2];
#pragma unroll
  for (int kk = 0; kk < 2; ++kk)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const long long nid =
            TOPO_IDX((ex + i) + (long long)nnx * ((ey + j) + (long long)nny * (ez + kk)), d.nodes());
        nu[kk][j][i] = {df_from_double(__ldg(v + 3 * nid))};
        nv[kk][j][i] = {df_from_double(__ldg(v + 3 * nid + 1))};
        nw[kk][j][i] = {df_from_double(__ldg(v + 3 * nid + 2))};
      }
  PairNum tu[7], tv[7], tw[7];
  wht_fwd(nu, tu);
  wht_fwd(nv, tv);
  wht_fwd(nw, tw);
  const float2 xe = __ldg(xdf + e);
  hex_khat(k, PairNum{{xe.x, xe.y}}, tu, tv, tw);
  wht_inv(tu, nu);
  wht_inv(tv, nv);
  wht_inv(tw, nw);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int i = hx_ox(a), j = hx_oy(a), kk = hx_oz(a);
    R[(long long)(a * 3 + 0) * m + e] = make_float2(nu[kk][j][i].v.h, nu[kk][j][i].v.l);
    R[(long long)(a * 3 + 1) * m + e] = make_float2(nv[kk][j][i].v.h, nv[kk][j][i].v.l);
    R[(long long)(a * 3 + 2) * m + e] = make_float2(nw[kk][j][i].v.h, nw[kk][j][i].v.l);
  }
}

__global__ void __launch_bounds__(kThreads) k_hex_gather_dot_df(Dims d, const float2* __restrict__ R,
                                                                const double* __restrict__ p,
                                                                double* __restrict__ q,
                                                                const uint8_t* __restrict__ fixed,
                                                                double* partials,
                                                                unsigned* counters,
                                                                CgScalars* sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc[rhs].done) return;
  const long long m = d.elems();
  const long long nodes = d.nodes();
  const long long n = nodes * 3;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  p += rhs * n;
  q += rhs * n;
  R += rhs * 24 * m;
  f2 part = {0.0f, 0.0f};
  if (node < nodes) {
    int i, j, kk;
    node_coords(node, d.nx + 1, d.ny + 1, 3, i, j, kk);
    f2 acc[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int s = 0; s < 8; ++s) {
      const int dx = s & 1, dy = (s >> 1) & 1, dz = s >> 2;
      const int ex = i - 1 + dx, ey = j - 1 + dy, ez = kk - 1 + dz;
      if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny || ez < 0 || ez >= d.nz) continue;
      const int lx = 1 - dx, ly = 1 - dy, lz = 1 - dz;
      const int loc = (ly ? (lx ? 2 : 3) : (lx ? 1 : 0)) + 4 * lz;
      const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
      if (!TOPO_IN(e, m)) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 r = __ldg(R + (long long)(loc * 3 + c) * m + e);
        acc[c] = df_add_nr(acc[c], f2{r.x, r.y});
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long id = 3 * node + c;
      if (!TOPO_IN(id, n)) continue;
      if (fixed[id]) acc[c] = f2{0.0f, 0.0f};
      q[id] = double_from_float(acc[c].h) + double_from_float(acc[c].l);
      part = df_add(part, df_mul(df_from_double(p[id]), acc[c]));
    }
  }
  const double bs = block_sum_hex(double_from_float(part.h) + double_from_float(part.l));
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
  s = block_sum_hex(s);
  if (threadIdx.x == 0) {
    CgScalars& S = sc[rhs];
    S.pq = s;
    const double alpha = S.ry / s;
    if (!(s > 0.0) || !isfinite(alpha)) {
      S.status = TOPO_E_BREAKDOWN;
      S.done = 1;
      S.alpha = 0.0;
    } else {
      S.alpha = alpha;
    }
    counters[rhs] = 0;
  }
}


// ---- Tile formulation: element forces through shared memory --------------------------------
// A block owns a tile of (TX - 1) x (TY - 1) node columns and a range of cz node planes.  Its TX x
// TY threads compute the elements of the tile plus one element row and column of halo (thread
// (tx, ty) the element whose lower-left-front node is its node), one element layer at a time,
// and write the 24 element forces to shared memory; after a barrier every thread with a node
// in its tile adds the forces of the four elements of that layer around the node.  Marching up
// the planes, a node plane is complete after the element layers below and above it: its forces
// are added in the order of k_hex_gather_dot (layer below, then layer above; x fastest), so q
// has the bits of the buffered form, without the 24 forces per element and right-hand side in
// global memory (192 bytes written and read again per element in FP64).  The halo elements are
// computed twice (in both tiles): the planner below picks the tile that minimises the element
// work with enough blocks.  Two force buffers alternate, so one barrier per layer suffices.
struct HexTile {
  int tx, ty, cz;          // threads per row, rows, node planes per block
  int tiles_x, tiles_y, zchunks;
};

__device__ __forceinline__ int tile_loc(int dx, int dy, int dz) {  // local node of the element
  const int lx = 1 - dx, ly = 1 - dy, lz = 1 - dz;
  return (ly ? (lx ? 2 : 3) : (lx ? 1 : 0)) + 4 * lz;
}

template <typename P>
struct HexTileElem;  // the force type stored in shared memory and the density input
template <>
struct HexTileElem<double> {
  using S = double;
  __device__ static double from_v(double v) { return v; }
  __device__ static double x_of(const void* x, long long e) {
    return __ldg(static_cast<const double*>(x) + e);
  }
  __device__ static S store(double a) { return a; }
  __device__ static double load(S a) { return a; }
};
template <>
struct HexTileElem<PairNum> {
  using S = float2;
  __device__ static PairNum from_v(double v) { return {df_from_double(v)}; }
  __device__ static PairNum x_of(const void* x, long long e) {
    const float2 v = __ldg(static_cast<const float2*>(x) + e);
    return {{v.x, v.y}};
  }
  __device__ static S store(PairNum a) { return make_float2(a.v.h, a.v.l); }
  __device__ static f2 load(S a) { return {a.x, a.y}; }
};

// Outer operator q = K(x) p (FP64 or float pairs), p^T q per block and alpha by the last block.
template <typename P>
__global__ void __launch_bounds__(512) k_hex_tile_outer(Dims d, HexTile tl, HexK<P> k,
                                                        const void* __restrict__ xin,
                                                        const double* __restrict__ v,
                                                        double* __restrict__ q,
                                                        const uint8_t* __restrict__ fixed,
                                                        double* partials, unsigned* counters,
                                                        CgScalars* sc) {
  using E = HexTileElem<P>;
  using S = typename E::S;
  pdl_prologue();
  const int rhs = blockIdx.z;
  if (sc[rhs].done) return;
  extern __shared__ float4 hex_tile_raw[];
  S* F = reinterpret_cast<S*>(hex_tile_raw);  // [2][24][TT]
  const int TT = tl.tx * tl.ty;
  const int t = threadIdx.x, tx = t % tl.tx, ty = t / tl.tx;
  const int bx = blockIdx.x % tl.tiles_x, by = blockIdx.x / tl.tiles_x;
  const int ex = bx * (tl.tx - 1) - 1 + tx, ey = by * (tl.ty - 1) - 1 + ty;
  const int nnx = d.nx + 1, nny = d.ny + 1, nnz = d.nz + 1;
  const int k0 = blockIdx.y * tl.cz, k1 = min(k0 + tl.cz, nnz);
  const long long m = d.elems(), nodes = d.nodes(), n = nodes * 3;
  v += rhs * n;
  q += rhs * n;
  const bool e_xy = ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny;
  // the node of this thread: (ex, ey), when the four elements around it are in the tile
  const bool own = tx >= 1 && ty >= 1 && ex < nnx && ey < nny;
  using Acc = decltype(E::load(S()));
  Acc acc[3];
  double part_d = 0.0;
  f2 part_f = {0.0f, 0.0f};
#pragma unroll
  for (int c = 0; c < 3; ++c) acc[c] = Acc{};
#pragma unroll 1
  for (int ez = k0 - 1; ez < k1; ++ez) {
    S* Fb = F + (size_t)((ez - k0 + 1) & 1) * 24 * TT;
    if (e_xy && ez >= 0 && ez < d.nz) {
      P nu[2][2][2], nv[2][2][2], nw[2][2][2];
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const long long nid =
            TOPO_IDX((ex + i) + (long long)nnx * ((ey + j) + (long long)nny * (ez + kk)), d.nodes());
            nu[kk][j][i] = E::from_v(__ldg(v + 3 * nid));
            nv[kk][j][i] = E::from_v(__ldg(v + 3 * nid + 1));
            nw[kk][j][i] = E::from_v(__ldg(v + 3 * nid + 2));
          }
      P tu[7], tv[7], tw[7];
      wht_fwd(nu, tu);
      wht_fwd(nv, tv);
      wht_fwd(nw, tw);
      const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
      hex_khat(k, E::x_of(xin, e), tu, tv, tw);
      wht_inv(tu, nu);
      wht_inv(tv, nv);
      wht_inv(tw, nw);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int i = hx_ox(a), j = hx_oy(a), kk = hx_oz(a);
        Fb[(a * 3 + 0) * TT + t] = E::store(nu[kk][j][i]);
        Fb[(a * 3 + 1) * TT + t] = E::store(nv[kk][j][i]);
        Fb[(a * 3 + 2) * TT + t] = E::store(nw[kk][j][i]);
      }
    }
    __syncthreads();
    if (own) {
      const bool lay = ez >= 0 && ez < d.nz;
      // plane ez: the forces of layer ez (above it) complete its sums
      if (ez >= k0) {
        if (lay) {
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int dx = s & 1, dy = s >> 1;
            const int gx = ex - 1 + dx, gy = ey - 1 + dy;
            if (gx < 0 || gx >= d.nx || gy < 0 || gy >= d.ny) continue;
            const int te = TOPO_IDX(t - (1 - dx) - (1 - dy) * tl.tx, TT);
            const int loc = tile_loc(dx, dy, 1);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              if constexpr (std::is_same<P, double>::value) acc[c] += Fb[(loc * 3 + c) * TT + te];
              else acc[c] = df_add_nr(acc[c], E::load(Fb[(loc * 3 + c) * TT + te]));
            }
          }
        }
        const long long node = ex + (long long)nnx * (ey + (long long)nny * ez);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const long long id = 3 * node + c;
          if (!TOPO_IN(id, n)) continue;
          if constexpr (std::is_same<P, double>::value) {
            const double out = fixed[id] ? 0.0 : acc[c];
            q[id] = out;
            part_d = fma(v[id], out, part_d);
          } else {
            if (fixed[id]) acc[c] = f2{0.0f, 0.0f};
            q[id] = double_from_float(acc[c].h) + double_from_float(acc[c].l);
            part_f = df_add(part_f, df_mul(df_from_double(v[id]), acc[c]));
          }
        }
      }
      // plane ez + 1: starts with the forces of layer ez (below it)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] = Acc{};
      if (lay && ez + 1 < k1) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int dx = s & 1, dy = s >> 1;
          const int gx = ex - 1 + dx, gy = ey - 1 + dy;
          if (gx < 0 || gx >= d.nx || gy < 0 || gy >= d.ny) continue;
          const int te = TOPO_IDX(t - (1 - dx) - (1 - dy) * tl.tx, TT);
          const int loc = tile_loc(dx, dy, 0);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            if constexpr (std::is_same<P, double>::value) acc[c] += Fb[(loc * 3 + c) * TT + te];
            else acc[c] = df_add_nr(acc[c], E::load(Fb[(loc * 3 + c) * TT + te]));
          }
        }
      }
    }
  }
  double part;
  if constexpr (std::is_same<P, double>::value) part = part_d;
  else part = double_from_float(part_f.h) + double_from_float(part_f.l);
  const double bs = block_sum_hex(part);
  const unsigned nb = gridDim.x * gridDim.y, bid = blockIdx.x + gridDim.x * blockIdx.y;
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[(long long)rhs * nb + bid] = bs;
    __threadfence();
    last = (atomicAdd(&counters[rhs], 1u) == nb - 1);
  }
  __syncthreads();
  if (!last) return;
  double s = 0.0;
  for (unsigned u = threadIdx.x; u < nb; u += blockDim.x) s += __ldcg(partials + (long long)rhs * nb + u);
  s = block_sum_hex(s);
  if (threadIdx.x == 0) {
    CgScalars& Sc = sc[rhs];
    Sc.pq = s;
    const double alpha = Sc.ry / s;
    if (!(s > 0.0) || !isfinite(alpha)) {
      Sc.status = TOPO_E_BREAKDOWN;
      Sc.done = 1;
      Sc.alpha = 0.0;
    } else {
      Sc.alpha = alpha;
    }
    counters[rhs] = 0;
  }
  (void)m;
}

// V-cycle operator on the finest level: mode 0 y = A v, 1 y = b - A v, 2 y = v + omega invd
// (b - A v).  DENSE: the element rows of K0 (shared memory) times the element's 24 values as
// FMA chains, and the node adds x_e t with one FMA per element: the arithmetic, and its order,
// of the node-parallel k_apply3_rhs, so the same bits.  Otherwise the Walsh-Hadamard form of
// the element (about 180 operations instead of 576 multiply-adds) with x_e in the coefficients
// and plain adds at the node (other roundings, the same operator).
// DOT 2 (MODE 2, the last smoothing sweep of the preconditioner): also r~^T y~ against the FP64
// CG residual rdot and, by the last block, beta = r~^T y~ / r^T y of Algorithm PCG (as the 2D
// sweeps form it).
template <typename T, int MODE, bool DENSE, int DOT = 0>
__global__ void __launch_bounds__(512) k_hex_tile_sweep(Dims d, HexTile tl, HexK<T> k,
                                                        const T* __restrict__ K0,
                                                        const T* __restrict__ x,
                                                        const T* __restrict__ v,
                                                        const T* __restrict__ b,
                                                        T* __restrict__ y,
                                                        const T* __restrict__ invd, T omega,
                                                        const uint8_t* __restrict__ fixed,
                                                        const CgScalars* __restrict__ sc,
                                                        const double* __restrict__ rdot = nullptr,
                                                        double* partials = nullptr,
                                                        unsigned* counters = nullptr) {
  pdl_prologue();
  const int rhs = blockIdx.z;
  if (sc && sc[rhs].done) return;
  double part = 0.0;
  extern __shared__ float4 hex_tile_raw[];
  const int TT = tl.tx * tl.ty;
  T* F = reinterpret_cast<T*>(hex_tile_raw);  // [2][24][TT]
  T* X = F + 2 * 24 * TT;                      // [2][TT] (DENSE)
  T* K0s = X + 2 * TT;                         // [576]  (DENSE)
  if (DENSE) {
    for (int u = threadIdx.x; u < 576; u += blockDim.x) K0s[u] = K0[u];
    __syncthreads();
  }
  const int t = threadIdx.x, tx = t % tl.tx, ty = t / tl.tx;
  const int bx = blockIdx.x % tl.tiles_x, by = blockIdx.x / tl.tiles_x;
  const int ex = bx * (tl.tx - 1) - 1 + tx, ey = by * (tl.ty - 1) - 1 + ty;
  const int nnx = d.nx + 1, nny = d.ny + 1, nnz = d.nz + 1;
  const int k0 = blockIdx.y * tl.cz, k1 = min(k0 + tl.cz, nnz);
  const long long n = d.nodes() * 3;
  v += rhs * n;
  y += rhs * n;
  if (MODE != 0) b += rhs * n;
  if (DOT == 2) rdot += rhs * n;
  const bool e_xy = ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny;
  const bool own = tx >= 1 && ty >= 1 && ex < nnx && ey < nny;
  T acc[3] = {T(0), T(0), T(0)};
#pragma unroll 1
  for (int ez = k0 - 1; ez < k1; ++ez) {
    const int buf = (ez - k0 + 1) & 1;
    T* Fb = F + (size_t)buf * 24 * TT;
    if (e_xy && ez >= 0 && ez < d.nz) {
      const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
      if (DENSE) {
        T ve[24];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const long long nid = TOPO_IDX(
              (ex + hx_ox(a)) + (long long)nnx * ((ey + hx_oy(a)) + (long long)nny * (ez + hx_oz(a))),
              d.nodes());
#pragma unroll
          for (int c = 0; c < 3; ++c) ve[a * 3 + c] = __ldg(v + 3 * nid + c);
        }
#pragma unroll 4
        for (int r = 0; r < 24; ++r) {
          T s = T(0);
#pragma unroll
          for (int qq = 0; qq < 24; ++qq) s = fma(K0s[r * 24 + qq], ve[qq], s);
          Fb[r * TT + t] = s;
        }
        X[buf * TT + t] = __ldg(x + e);
      } else {
        T nu[2][2][2], nv[2][2][2], nw[2][2][2];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
#pragma unroll
          for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
              const long long nid =
            TOPO_IDX((ex + i) + (long long)nnx * ((ey + j) + (long long)nny * (ez + kk)), d.nodes());
              nu[kk][j][i] = __ldg(v + 3 * nid);
              nv[kk][j][i] = __ldg(v + 3 * nid + 1);
              nw[kk][j][i] = __ldg(v + 3 * nid + 2);
            }
        T tu[7], tv[7], tw[7];
        wht_fwd(nu, tu);
        wht_fwd(nv, tv);
        wht_fwd(nw, tw);
        hex_khat(k, __ldg(x + e), tu, tv, tw);
        wht_inv(tu, nu);
        wht_inv(tv, nv);
        wht_inv(tw, nw);
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int i = hx_ox(a), j = hx_oy(a), kk = hx_oz(a);
          Fb[(a * 3 + 0) * TT + t] = nu[kk][j][i];
          Fb[(a * 3 + 1) * TT + t] = nv[kk][j][i];
          Fb[(a * 3 + 2) * TT + t] = nw[kk][j][i];
        }
      }
    }
    __syncthreads();
    if (own) {
      const bool lay = ez >= 0 && ez < d.nz;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        // half 0: layer ez completes plane ez (dz = 1); half 1: it starts plane ez + 1 (dz = 0)
        const int dz = 1 - half;
        if (half == 0 && ez < k0) continue;
        if (half == 1 && ez + 1 >= k1) continue;
        if (lay) {
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int dx = s & 1, dy = s >> 1;
            const int gx = ex - 1 + dx, gy = ey - 1 + dy;
            if (gx < 0 || gx >= d.nx || gy < 0 || gy >= d.ny) continue;
            const int te = TOPO_IDX(t - (1 - dx) - (1 - dy) * tl.tx, TT);
            const int loc = tile_loc(dx, dy, dz);
            const T xe = DENSE ? X[buf * TT + te] : T(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const T f = Fb[(loc * 3 + c) * TT + te];
              acc[c] = DENSE ? fma(xe, f, acc[c]) : acc[c] + f;
            }
          }
        }
        if (half == 0) {
          const long long node = ex + (long long)nnx * (ey + (long long)nny * ez);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const long long id = 3 * node + c;
            if (!TOPO_IN(id, n)) continue;
            T out;
            if (fixed[id]) out = T(0);
            else if (MODE == 0) out = acc[c];
            else if (MODE == 1) out = node_out<1, T>(acc[c], T(0), __ldg(b + id), T(0), omega);
            else out = node_out<2, T>(acc[c], __ldg(v + id), __ldg(b + id), invd[id], omega);
            y[id] = out;
            if (DOT == 2) part = fma(__ldg(rdot + id), double_of(out), part);
            acc[c] = T(0);
          }
        }
      }
    }
  }
  if (DOT == 2) {  // beta by the last block, as the 2D sweeps finish it
    const double bs = block_sum_hex(part);
    const unsigned nb = gridDim.x * gridDim.y, bid = blockIdx.x + gridDim.x * blockIdx.y;
    __shared__ bool last;
    if (threadIdx.x == 0) {
      partials[(long long)rhs * nb + bid] = bs;
      __threadfence();
      last = (atomicAdd(&counters[rhs], 1u) == nb - 1);
    }
    __syncthreads();
    if (!last) return;
    double s2 = 0.0;
    for (unsigned u = threadIdx.x; u < nb; u += blockDim.x) s2 += __ldcg(partials + (long long)rhs * nb + u);
    s2 = block_sum_hex(s2);
    if (threadIdx.x == 0) {
      CgScalars& S = const_cast<CgScalars&>(sc[rhs]);
      const double beta = s2 / S.ry;
      S.ry_new = s2;
      S.beta = beta;
      S.ry = s2;
      if (!isfinite(beta)) {
        S.status = TOPO_E_BREAKDOWN;
        S.done = 1;
      }
      counters[rhs] = 0;
    }
  }
}


// ---- Tensor-core form of the dense tile sweep (evaluation) ----------------------------------
// The element rows of K0 times the element vectors as a warp-level matrix product on the tensor
// cores: for the 32 elements of a warp, T[24 x 32] = K0[24 x 24] V[24 x 32] with mma.sync
// m16n8k8 in TF32, K0 and V split into TF32 high and low parts and the three products hi hi,
// hi lo, lo hi accumulated in FP32 (about the accuracy of FP32 products; other roundings than
// the FMA chains of the dense form).  Rows 24..31 of the second M tile are zero.  The element
// vectors reach the B fragments through a per-warp shared-memory transpose (stride 40 words:
// the eight rows of a fragment fall in distinct banks); the products go to the force buffer of
// the tile skeleton, and the node phase is that of the dense form (x_e t added by FMA).
__device__ __forceinline__ unsigned tf32_rna(float f) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}

__device__ __forceinline__ void mma_tf32(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kTcStride = 40;  // words per row of the per-warp transpose buffer

template <int MODE>
__global__ void __launch_bounds__(512) k_hex_tile_sweep_tc(Dims d, HexTile tl,
                                                           const float* __restrict__ K0,
                                                           const float* __restrict__ x,
                                                           const float* __restrict__ v,
                                                           const float* __restrict__ b,
                                                           float* __restrict__ y,
                                                           const float* __restrict__ invd,
                                                           float omega,
                                                           const uint8_t* __restrict__ fixed,
                                                           const CgScalars* __restrict__ sc) {
  pdl_prologue();
  const int rhs = blockIdx.z;
  if (sc && sc[rhs].done) return;
  extern __shared__ float4 hex_tile_raw[];
  const int TT = tl.tx * tl.ty;
  float* F = reinterpret_cast<float*>(hex_tile_raw);  // [2][24][TT]
  float* X = F + 2 * 24 * TT;                          // [2][TT]
  float* Vs = X + 2 * TT;                              // [warps][24][kTcStride]
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  float* Vw = Vs + warp * 24 * kTcStride;
  // A fragments of K0 (hi, lo): m tile mt (rows 16 mt + gid, + 8), k step ks (cols 8 ks + tig, + 4)
  unsigned ah[2][3][4], al[2][3][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int ks = 0; ks < 3; ++ks)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = 16 * mt + gid + ((r & 1) ? 8 : 0), col = 8 * ks + tig + ((r & 2) ? 4 : 0);
        const float a = row < 24 ? __ldg(K0 + row * 24 + col) : 0.0f;
        ah[mt][ks][r] = tf32_rna(a);
        al[mt][ks][r] = tf32_rna(a - __uint_as_float(ah[mt][ks][r]));
      }
  const int tx = t % tl.tx, ty = t / tl.tx;
  const int bx = blockIdx.x % tl.tiles_x, by = blockIdx.x / tl.tiles_x;
  const int ex = bx * (tl.tx - 1) - 1 + tx, ey = by * (tl.ty - 1) - 1 + ty;
  const int nnx = d.nx + 1, nny = d.ny + 1, nnz = d.nz + 1;
  const int k0 = blockIdx.y * tl.cz, k1 = min(k0 + tl.cz, nnz);
  const long long n = d.nodes() * 3;
  v += rhs * n;
  y += rhs * n;
  if (MODE != 0) b += rhs * n;
  const bool e_xy = ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny;
  const bool own = tx >= 1 && ty >= 1 && ex < nnx && ey < nny;
  float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll 1
  for (int ez = k0 - 1; ez < k1; ++ez) {
    const int buf = (ez - k0 + 1) & 1;
    float* Fb = F + (size_t)buf * 24 * TT;
    const bool live = e_xy && ez >= 0 && ez < d.nz;
    // the element vector of this lane (zeros for no element) into the warp's transpose buffer
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      long long nid = 0;
      if (live)
        nid = TOPO_IDX((ex + hx_ox(a)) + (long long)nnx * ((ey + hx_oy(a)) + (long long)nny * (ez + hx_oz(a))),
                       d.nodes());
#pragma unroll
      for (int c = 0; c < 3; ++c) Vw[(a * 3 + c) * kTcStride + lane] = live ? __ldg(v + 3 * nid + c) : 0.0f;
    }
    if (live) X[buf * TT + t] = __ldg(x + ex + (long long)d.nx * (ey + (long long)d.ny * ez));
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      float cacc[2][4] = {{0.0f, 0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
#pragma unroll
      for (int ks = 0; ks < 3; ++ks) {
        const float v0 = Vw[(8 * ks + tig) * kTcStride + 8 * nt + gid];
        const float v1 = Vw[(8 * ks + tig + 4) * kTcStride + 8 * nt + gid];
        const unsigned bh0 = tf32_rna(v0), bh1 = tf32_rna(v1);
        const unsigned bl0 = tf32_rna(v0 - __uint_as_float(bh0)),
                       bl1 = tf32_rna(v1 - __uint_as_float(bh1));
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma_tf32(cacc[mt], al[mt][ks], bh0, bh1);
          mma_tf32(cacc[mt], ah[mt][ks], bl0, bl1);
          mma_tf32(cacc[mt], ah[mt][ks], bh0, bh1);
        }
      }
      // D (row 16 mt + gid (+ 8), element 8 nt + 2 tig (+ 1)) into the force buffer
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int row = 16 * mt + gid + ((r & 2) ? 8 : 0);
          const int el = 32 * warp + 8 * nt + 2 * tig + (r & 1);
          if (row < 24) Fb[row * TT + el] = cacc[mt][r];
        }
    }
    __syncthreads();
    if (own) {
      const bool lay = ez >= 0 && ez < d.nz;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int dz = 1 - half;
        if (half == 0 && ez < k0) continue;
        if (half == 1 && ez + 1 >= k1) continue;
        if (lay) {
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int dx = s & 1, dy = s >> 1;
            const int gx = ex - 1 + dx, gy = ey - 1 + dy;
            if (gx < 0 || gx >= d.nx || gy < 0 || gy >= d.ny) continue;
            const int te = TOPO_IDX(t - (1 - dx) - (1 - dy) * tl.tx, TT);
            const int loc = tile_loc(dx, dy, dz);
            const float xe = X[buf * TT + te];
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[c] = fmaf(xe, Fb[(loc * 3 + c) * TT + te], acc[c]);
          }
        }
        if (half == 0) {
          const long long node = ex + (long long)nnx * (ey + (long long)nny * ez);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const long long id = 3 * node + c;
            if (!TOPO_IN(id, n)) continue;
            float out;
            if (fixed[id]) out = 0.0f;
            else if (MODE == 0) out = acc[c];
            else if (MODE == 1) out = node_out<1, float>(acc[c], 0.0f, __ldg(b + id), 0.0f, omega);
            else out = node_out<2, float>(acc[c], __ldg(v + id), __ldg(b + id), invd[id], omega);
            y[id] = out;
            acc[c] = 0.0f;
          }
        }
      }
    }
    __syncwarp();  // (the transpose buffer is rewritten by the next layer)
  }
}

}  // namespace

bool hex_coefficients(const double* K0, HexCoef& c) {
  // T: row (comp * 8 + mode), column (node * 3 + comp); modes 1, xi, eta, zeta, xieta, etazeta,
  // xizeta, xietazeta
  const int ox[8] = {0, 1, 1, 0, 0, 1, 1, 0}, oy[8] = {0, 0, 1, 1, 0, 0, 1, 1},
            oz[8] = {0, 0, 0, 0, 1, 1, 1, 1};
  double H[8][8];
  for (int a = 0; a < 8; ++a) {
    const double xi = 2 * ox[a] - 1, eta = 2 * oy[a] - 1, zeta = 2 * oz[a] - 1;
    const double md[8] = {1, xi, eta, zeta, xi * eta, eta * zeta, xi * zeta, xi * eta * zeta};
    for (int mm = 0; mm < 8; ++mm) H[mm][a] = md[mm];
  }
  std::vector<double> T(24 * 24, 0.0);
  for (int cc = 0; cc < 3; ++cc)
    for (int mm = 0; mm < 8; ++mm)
      for (int a = 0; a < 8; ++a) T[(cc * 8 + mm) * 24 + a * 3 + cc] = H[mm][a];
  // Khat = T K0 T^T / 64 (T^-1 = T^T / 8)
  std::vector<double> TK(24 * 24, 0.0), Kh(24 * 24, 0.0);
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) {
      double acc = 0.0;
      for (int l = 0; l < 24; ++l) acc += T[i * 24 + l] * K0[l * 24 + j];
      TK[i * 24 + j] = acc;
    }
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) {
      double acc = 0.0;
      for (int l = 0; l < 24; ++l) acc += TK[i * 24 + l] * T[j * 24 + l];
      Kh[i * 24 + j] = acc / 64.0;
    }
  auto at = [&](int c1, int m1, int c2, int m2) { return Kh[(c1 * 8 + m1) * 24 + c2 * 8 + m2]; };
  c.a = at(0, 1, 0, 1);
  c.b = at(0, 1, 1, 2);
  c.s = at(0, 2, 0, 2);
  c.p = at(0, 4, 0, 4);
  c.q = at(0, 4, 2, 5);
  c.d = at(0, 5, 0, 5);
  c.e = at(0, 5, 1, 6);
  c.h = at(0, 7, 0, 7);
  // the structured Khat from the eight numbers, then T^T Khat T against K0
  std::vector<double> Ks(24 * 24, 0.0);
  auto set = [&](int c1, int m1, int c2, int m2, double val) {
    Ks[(c1 * 8 + m1) * 24 + c2 * 8 + m2] = val;
    Ks[(c2 * 8 + m2) * 24 + c1 * 8 + m1] = val;
  };
  for (int cc = 0; cc < 3; ++cc) set(cc, 1 + cc, cc, 1 + cc, c.a);
  set(0, 1, 1, 2, c.b);
  set(0, 1, 2, 3, c.b);
  set(1, 2, 2, 3, c.b);
  const int sh[3][4] = {{0, 2, 1, 1}, {0, 3, 2, 1}, {1, 3, 2, 2}};  // (u,eta)(v,xi) etc.
  for (auto& z : sh) {
    set(z[0], z[1], z[0], z[1], c.s);
    set(z[2], z[3], z[2], z[3], c.s);
    set(z[0], z[1], z[2], z[3], c.s);
  }
  const int pr[3][4] = {{0, 4, 2, 5}, {0, 6, 1, 5}, {1, 4, 2, 6}};  // bilinear pairs
  for (auto& z : pr) {
    set(z[0], z[1], z[0], z[1], c.p);
    set(z[2], z[3], z[2], z[3], c.p);
    set(z[0], z[1], z[2], z[3], c.q);
  }
  const int tr[3][2] = {{0, 5}, {1, 6}, {2, 4}};  // (u,etazeta) (v,xizeta) (w,xieta)
  for (int i = 0; i < 3; ++i) {
    set(tr[i][0], tr[i][1], tr[i][0], tr[i][1], c.d);
    for (int j = i + 1; j < 3; ++j) set(tr[i][0], tr[i][1], tr[j][0], tr[j][1], c.e);
  }
  for (int cc = 0; cc < 3; ++cc) set(cc, 7, cc, 7, c.h);
  double err = 0.0, scale = 0.0;
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) {
      double acc = 0.0;
      for (int l = 0; l < 24; ++l)
        for (int r = 0; r < 24; ++r) acc += T[l * 24 + i] * Ks[l * 24 + r] * T[r * 24 + j];
      err = std::max(err, std::fabs(acc - K0[i * 24 + j]));
      scale = std::max(scale, std::fabs(K0[i * 24 + j]));
    }
  return err <= 1e-13 * scale;
}

cudaError_t launch_hex_apply_dot(const Dims& d, const HexCoef& c, const double* x, const double* v,
                                 double* y, const uint8_t* fixed, int nrhs, double* R,
                                 double* partials, unsigned* counters, CgScalars* sc,
                                 cudaStream_t st) {
  const HexK<double> k{c.a, c.b, c.s, c.p, c.q, c.d, c.e, c.h};
  topo::launch(k_hex_elem, dim3(blocks_for(d.elems()), nrhs), kThreads, 0, st, d, k, x, v, R,
               (const CgScalars*)sc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  topo::launch(k_hex_gather_dot, dim3(blocks_for(d.nodes()), nrhs), kThreads, 0, st, d,
               (const double*)R, v, y, fixed, partials, counters, sc);
  return cudaGetLastError();
}

cudaError_t launch_hex_apply_dot_df(const Dims& d, const HexCoef& c, const float2* xdf,
                                    const double* v, double* y, const uint8_t* fixed, int nrhs,
                                    double* R, double* partials, unsigned* counters, CgScalars* sc,
                                    cudaStream_t st) {
  const HexK<PairNum> k{{df_const(c.a)}, {df_const(c.b)}, {df_const(c.s)}, {df_const(c.p)},
                        {df_const(c.q)}, {df_const(c.d)}, {df_const(c.e)}, {df_const(c.h)}};
  float2* Rp = reinterpret_cast<float2*>(R);  // (pairs in the FP64 buffer: the same bytes)
  topo::launch(k_hex_elem_df, dim3(blocks_for(d.elems()), nrhs), kThreads, 0, st, d, k, xdf, v,
               Rp, (const CgScalars*)sc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  topo::launch(k_hex_gather_dot_df, dim3(blocks_for(d.nodes()), nrhs), kThreads, 0, st, d,
               (const float2*)Rp, v, y, fixed, partials, counters, sc);
  return cudaGetLastError();
}


// Tile plan: the (TX, TY) with at most max_threads threads (a multiple of 32) and the number of
// z chunks that minimise the element work (halo included) with at least `target` blocks.
HexTile hex_tile_plan(const Dims& d, int nrhs, int max_threads, int target) {
  HexTile best = {};
  double best_work = 0.0;
  const int nnx = d.nx + 1, nny = d.ny + 1, nnz = d.nz + 1;
  for (int ty = 2; ty <= 32; ++ty)
    for (int tx = 4; tx <= 128; ++tx) {
      const int th = tx * ty;
      if (th % 32 || th > max_threads || th < 64) continue;
      const int tiles_x = (nnx + tx - 2) / (tx - 1), tiles_y = (nny + ty - 2) / (ty - 1);
      const long long tiles = (long long)tiles_x * tiles_y;
      if (tiles > 65535) continue;
      long long zc = (target + tiles * nrhs - 1) / (tiles * nrhs);
      zc = std::max(1LL, std::min<long long>(zc, nnz));
      const int cz = (int)((nnz + zc - 1) / zc);
      zc = (nnz + cz - 1) / cz;
      if (tiles * zc > (long long)kMaxRedValues * kRedBlocks) continue;
      const double work = (double)tiles * th * (double)zc * (cz + 1);
      if (best.tx == 0 || work < best_work * 0.999 ||
          (work <= best_work * 1.001 && th > best.tx * best.ty)) {
        best = {tx, ty, cz, tiles_x, tiles_y, (int)zc};
        best_work = work;
      }
    }
  return best;
}

template <typename K>
static cudaError_t hex_tile_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

constexpr int kHexTileOuterThreads = 256;  // (the pair element product keeps ~130 registers)
constexpr int kHexTileSweepThreads = 512;

cudaError_t prepare_hex_tile_kernels() {
  cudaError_t e = hex_tile_smem(k_hex_tile_outer<double>, 2 * 24 * kHexTileOuterThreads * 8);
  if (e == cudaSuccess) e = hex_tile_smem(k_hex_tile_outer<PairNum>, 2 * 24 * kHexTileOuterThreads * 8);
#define TOPO_HT_PREP(T, MODE)                                                                      \
  if (e == cudaSuccess)                                                                            \
    e = hex_tile_smem(k_hex_tile_sweep<T, MODE, true>,                                             \
                      (2 * 24 * kHexTileSweepThreads + 2 * kHexTileSweepThreads + 576) * sizeof(T)); \
  if (e == cudaSuccess)                                                                            \
    e = hex_tile_smem(k_hex_tile_sweep<T, MODE, false>,                                            \
                      (2 * 24 * kHexTileSweepThreads + 2 * kHexTileSweepThreads + 576) * sizeof(T));
  TOPO_HT_PREP(float, 0)
  TOPO_HT_PREP(float, 1)
  TOPO_HT_PREP(float, 2)
  TOPO_HT_PREP(double, 0)
  TOPO_HT_PREP(double, 1)
  TOPO_HT_PREP(double, 2)
#undef TOPO_HT_PREP
#define TOPO_HT_PREPB(T)                                                                           \
  if (e == cudaSuccess)                                                                            \
    e = hex_tile_smem(k_hex_tile_sweep<T, 2, true, 2>,                                             \
                      (2 * 24 * kHexTileSweepThreads + 2 * kHexTileSweepThreads + 576) * sizeof(T)); \
  if (e == cudaSuccess)                                                                            \
    e = hex_tile_smem(k_hex_tile_sweep<T, 2, false, 2>,                                            \
                      (2 * 24 * kHexTileSweepThreads + 2 * kHexTileSweepThreads + 576) * sizeof(T));
  TOPO_HT_PREPB(float)
  TOPO_HT_PREPB(double)
#undef TOPO_HT_PREPB
  const size_t tc_smem = (2 * 24 * kHexTileSweepThreads + 2 * kHexTileSweepThreads +
                          (kHexTileSweepThreads / 32) * 24 * kTcStride) * sizeof(float);
  if (e == cudaSuccess) e = hex_tile_smem(k_hex_tile_sweep_tc<0>, tc_smem);
  if (e == cudaSuccess) e = hex_tile_smem(k_hex_tile_sweep_tc<1>, tc_smem);
  if (e == cudaSuccess) e = hex_tile_smem(k_hex_tile_sweep_tc<2>, tc_smem);
  return e;
}

cudaError_t launch_hex_tile_apply_dot(const Dims& d, const HexCoef& c, const void* x, bool pairs,
                                      const double* v, double* y, const uint8_t* fixed, int nrhs,
                                      double* partials, unsigned* counters, CgScalars* sc,
                                      cudaStream_t st) {
  const HexTile tl = hex_tile_plan(d, nrhs, kHexTileOuterThreads, 152 * 6);
  if (tl.tx == 0) return cudaErrorInvalidConfiguration;
  const dim3 grid(tl.tiles_x * tl.tiles_y, tl.zchunks, nrhs);
  const size_t smem = (size_t)2 * 24 * tl.tx * tl.ty * 8;
  if (pairs) {
    const HexK<PairNum> k{{df_const(c.a)}, {df_const(c.b)}, {df_const(c.s)}, {df_const(c.p)},
                          {df_const(c.q)}, {df_const(c.d)}, {df_const(c.e)}, {df_const(c.h)}};
    topo::launch(k_hex_tile_outer<PairNum>, grid, tl.tx * tl.ty, smem, st, d, tl, k, x, v, y,
                 fixed, partials, counters, sc);
  } else {
    const HexK<double> k{c.a, c.b, c.s, c.p, c.q, c.d, c.e, c.h};
    topo::launch(k_hex_tile_outer<double>, grid, tl.tx * tl.ty, smem, st, d, tl, k, x, v, y,
                 fixed, partials, counters, sc);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hex_tile_sweep(const Dims& d, int mode, int form, const HexCoef& c,
                                  const T* K0, const T* x, const T* v, const T* b, T* y,
                                  const T* invd, T omega, const uint8_t* fixed, int nrhs,
                                  const CgScalars* sc, cudaStream_t st) {
  const bool dense = form == 1;
  const int maxt = sizeof(T) == 8 ? 256 : kHexTileSweepThreads;
  const HexTile tl = hex_tile_plan(d, nrhs, maxt, 152 * 4);
  if (tl.tx == 0) return cudaErrorInvalidConfiguration;
  const dim3 grid(tl.tiles_x * tl.tiles_y, tl.zchunks, nrhs);
  const int TT = tl.tx * tl.ty;
  if constexpr (sizeof(T) == 4) {
    if (form == 2) {  // the tensor-core form
      const size_t smem = (size_t)(2 * 24 * TT + 2 * TT + (TT / 32) * 24 * kTcStride) * sizeof(float);
      if (mode == 0)
        topo::launch(k_hex_tile_sweep_tc<0>, grid, TT, smem, st, d, tl, K0, x, v, b, y, invd, omega,
                     fixed, sc);
      else if (mode == 1)
        topo::launch(k_hex_tile_sweep_tc<1>, grid, TT, smem, st, d, tl, K0, x, v, b, y, invd, omega,
                     fixed, sc);
      else if (mode == 2)
        topo::launch(k_hex_tile_sweep_tc<2>, grid, TT, smem, st, d, tl, K0, x, v, b, y, invd, omega,
                     fixed, sc);
      else
        return cudaErrorInvalidValue;
      return cudaGetLastError();
    }
  }
  if (form == 2) return cudaErrorInvalidValue;  // (FP32 only)
  const size_t smem = (size_t)(2 * 24 * TT + (dense ? 2 * TT + 576 : 0)) * sizeof(T);
  const HexK<T> k{(T)c.a, (T)c.b, (T)c.s, (T)c.p, (T)c.q, (T)c.d, (T)c.e, (T)c.h};
#define TOPO_HT(MODE, DENSE)                                                                     \
  topo::launch(k_hex_tile_sweep<T, MODE, DENSE>, grid, TT, smem, st, d, tl, k, K0, x, v, b, y, \
               invd, omega, fixed, sc, (const double*)nullptr, (double*)nullptr,                 \
               (unsigned*)nullptr)
  if (dense) {
    if (mode == 0) TOPO_HT(0, true);
    else if (mode == 1) TOPO_HT(1, true);
    else if (mode == 2) TOPO_HT(2, true);
    else return cudaErrorInvalidValue;
  } else {
    if (mode == 0) TOPO_HT(0, false);
    else if (mode == 1) TOPO_HT(1, false);
    else if (mode == 2) TOPO_HT(2, false);
    else return cudaErrorInvalidValue;
  }
#undef TOPO_HT
  return cudaGetLastError();
}

// The last smoothing sweep with r~^T y~ and beta (DOT 2): forms 0 (Walsh-Hadamard) and 1 (dense).
template <typename T>
cudaError_t launch_hex_tile_sweep_beta(const Dims& d, int form, const HexCoef& c, const T* K0,
                                       const T* x, const T* v, const T* b, T* y, const T* invd,
                                       T omega, const uint8_t* fixed, int nrhs, CgScalars* sc,
                                       const double* rdot, double* partials, unsigned* counters,
                                       cudaStream_t st) {
  const int maxt = sizeof(T) == 8 ? 256 : kHexTileSweepThreads;
  const HexTile tl = hex_tile_plan(d, nrhs, maxt, 152 * 4);
  if (tl.tx == 0) return cudaErrorInvalidConfiguration;
  const dim3 grid(tl.tiles_x * tl.tiles_y, tl.zchunks, nrhs);
  const int TT = tl.tx * tl.ty;
  const bool dense = form == 1;
  const size_t smem = (size_t)(2 * 24 * TT + (dense ? 2 * TT + 576 : 0)) * sizeof(T);
  const HexK<T> k{(T)c.a, (T)c.b, (T)c.s, (T)c.p, (T)c.q, (T)c.d, (T)c.e, (T)c.h};
  if (dense)
    topo::launch(k_hex_tile_sweep<T, 2, true, 2>, grid, TT, smem, st, d, tl, k, K0, x, v, b, y, invd,
                 omega, fixed, (const CgScalars*)sc, rdot, partials, counters);
  else
    topo::launch(k_hex_tile_sweep<T, 2, false, 2>, grid, TT, smem, st, d, tl, k, K0, x, v, b, y,
                 invd, omega, fixed, (const CgScalars*)sc, rdot, partials, counters);
  return cudaGetLastError();
}
template cudaError_t launch_hex_tile_sweep_beta<float>(const Dims&, int, const HexCoef&, const float*,
                                                       const float*, const float*, const float*,
                                                       float*, const float*, float, const uint8_t*,
                                                       int, CgScalars*, const double*, double*,
                                                       unsigned*, cudaStream_t);
template cudaError_t launch_hex_tile_sweep_beta<double>(const Dims&, int, const HexCoef&,
                                                        const double*, const double*,
                                                        const double*, const double*, double*,
                                                        const double*, double, const uint8_t*, int,
                                                        CgScalars*, const double*, double*,
                                                        unsigned*, cudaStream_t);

template cudaError_t launch_hex_tile_sweep<float>(const Dims&, int, int, const HexCoef&,
                                                  const float*, const float*, const float*,
                                                  const float*, float*, const float*, float,
                                                  const uint8_t*, int, const CgScalars*,
                                                  cudaStream_t);
template cudaError_t launch_hex_tile_sweep<double>(const Dims&, int, int, const HexCoef&,
                                                   const double*, const double*, const double*,
                                                   const double*, double*, const double*, double,
                                                   const uint8_t*, int, const CgScalars*,
                                                   cudaStream_t);

}  // namespace topo
