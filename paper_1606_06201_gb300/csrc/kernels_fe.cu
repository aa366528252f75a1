// Finite-element kernels on structured grids: the operator K(x) v = sum_e x_e L_e^T K0 L_e v on
// the finest level (matrix-free, element by element: Eq. (to), Sec. 7), the same with assembled
// Galerkin element matrices on coarse levels (Sec. 5.1), damped Jacobi sweeps (the smoother opt()
// of Algorithm MG), the bilinear/trilinear transfers of Sec. 7 (prolongation stencil
// [1/4 1/2 1/4; 1/2 1 1/2; 1/4 1/2 1/4], restriction = transpose) and element energies.
//
// All operators are gather formulations: one thread owns one node and sums the contributions of
// the 4 (2D) or 8 (3D) elements around it in a fixed order, so results are deterministic and no
// atomics are used.  Fixed DOFs are masked: their outputs are 0.
#include "topo_internal.cuh"

namespace topo {

namespace {

template <int DIM>
struct Elem {
  static constexpr int NN = DIM == 2 ? 4 : 8;       // nodes per element
  static constexpr int NE = NN * DIM;               // DOFs per element
};

// Local node offsets: counter-clockwise (0,0) (1,0) (1,1) (0,1), bottom face then top face.
__device__ __forceinline__ int loc_ox(int a) { return ((a & 3) == 1 || (a & 3) == 2) ? 1 : 0; }
__device__ __forceinline__ int loc_oy(int a) { return ((a & 3) >= 2) ? 1 : 0; }
__device__ __forceinline__ int loc_oz(int a) { return a >> 2; }
__device__ __forceinline__ int loc_of(int lx, int ly, int lz) {
  return (ly ? (lx ? 2 : 3) : (lx ? 1 : 0)) + 4 * lz;
}

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Load of a vector entry: through the read-only path (ldg), or, when COH, from L2 (ld.global.cg):
// the fused coarse-level kernel reads vectors that other blocks of its cluster wrote earlier in
// the same launch, which the non-coherent read-only path may not see.
template <bool COH, typename T>
__device__ __forceinline__ T vld(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}

// Entries of the vector a sweep multiplies, by DOF index.  VLoad reads a stored vector; VJac0 forms
// the first Jacobi sweep from zero, omega D^{-1} b (as apply_node MODE 3), so that the fused mode 4
// of apply_node sweeps on it without storing it: the same arithmetic in the same order.
template <bool COH, typename T>
struct VLoad {
  const T* v;
  __device__ __forceinline__ T operator()(long long i) const { return vld<COH>(v + i); }
};

template <bool COH, typename T>
struct VJac0 {
  const T* b;
  const T* invd;
  const uint8_t* fixed;
  T omega;
  __device__ __forceinline__ T operator()(long long i) const {
    return fixed[i] ? T(0) : mul_rn(mul_rn(omega, invd[i]), vld<COH>(b + i));
  }
};

// Sum over the elements around node (i,j,k) of rows (loc*DIM + c) of the element matrix times
// the element's DOF values.  FINE: element matrix x_e K0; otherwise the Galerkin element matrices
// stored entry-major, Ae[(row * NE + col) * m + e], so that a warp reading one entry of 32
// consecutive elements reads contiguous memory.
template <int DIM, typename T, bool FINE, typename VIn>
__device__ __forceinline__ void node_apply(const Dims& d, int i, int j, int k,
                                           const T* __restrict__ K0, const T* __restrict__ x,
                                           const T* __restrict__ Ae, const VIn& vin,
                                           T acc[DIM]) {
  constexpr int NN = Elem<DIM>::NN, NE = Elem<DIM>::NE;
  const int nnx = d.nx + 1, nny = d.ny + 1;
  const long long m = d.elems();
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
  if constexpr (DIM == 2 && !FINE) {
    // Coarse 2D levels are latency-bound: all 64 matrix entries and 32 vector entries of the
    // four adjacent elements are loaded before any is used (a missing element reads element 0
    // and node 0 and is not accumulated).
    T a[4][16], ve[4][8];
    bool ok[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int dx = s & 1, dy = s >> 1;
      const int ex = i - 1 + dx, ey = j - 1 + dy;
      ok[s] = ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny;
      const int loc = loc_of(1 - dx, 1 - dy, 0);
      const long long e = ok[s] ? TOPO_IDX(ex + (long long)d.nx * ey, m) : 0;
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int q = 0; q < 8; ++q)
          a[s][c * 8 + q] = ldg(Ae + (long long)((loc * 2 + c) * 8 + q) * m + e);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const long long nid =
            ok[s] ? TOPO_IDX((ex + loc_ox(b)) + (long long)nnx * (ey + loc_oy(b)), d.nodes()) : 0;
        ve[s][2 * b] = vin(2 * nid);
        ve[s][2 * b + 1] = vin(2 * nid + 1);
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (!ok[s]) continue;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        T t = T(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) t = fma(a[s][c * 8 + q], ve[s][q], t);
        acc[c] += t;
      }
    }
  } else {
#pragma unroll 1
  for (int s = 0; s < NN; ++s) {
    const int dx = s & 1, dy = (s >> 1) & 1, dz = (DIM == 3) ? (s >> 2) : 0;
    const int ex = i - 1 + dx, ey = j - 1 + dy, ez = (DIM == 3) ? k - 1 + dz : 0;
    if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny) continue;
    if (DIM == 3 && (ez < 0 || ez >= d.nz)) continue;
    const int loc = loc_of(1 - dx, 1 - dy, DIM == 3 ? 1 - dz : 0);
    const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
    if (!TOPO_IN(e, m)) continue;
    T ve[NE];
#pragma unroll
    for (int a = 0; a < NN; ++a) {
      const long long nid = TOPO_IDX((ex + loc_ox(a)) + (long long)nnx * ((ey + loc_oy(a)) +
                                                                          (long long)nny * (ez + loc_oz(a))),
                                     d.nodes());
#pragma unroll
      for (int c = 0; c < DIM; ++c) ve[a * DIM + c] = vin(DIM * nid + c);
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      T t = T(0);
      if (FINE) {
        const T* row = K0 + (loc * DIM + c) * NE;
#pragma unroll
        for (int q = 0; q < NE; ++q) t = fma(ldg(row + q), ve[q], t);
        acc[c] = fma(ldg(x + e), t, acc[c]);
      } else {
        const T* row = Ae + (long long)((loc * DIM + c) * NE) * m + e;
#pragma unroll
        for (int q = 0; q < NE; ++q) t = fma(ldg(row + (long long)q * m), ve[q], t);
        acc[c] += t;
      }
    }
  }
  }
}

// mode 0: y = A v;  1: y = b - A v;  2: y = v + omega invd (b - A v);  3: y = omega invd b,
// for the DIM entries of one node (v, b, y of the right-hand side at hand; w: arrow column).
// MODE 4: the sweep on VJac0 (the first two sweeps from zero).  vin supplies the swept vector.
template <int DIM, typename T, int MODE, bool FINE, bool COH, typename VIn>
__device__ __forceinline__ void apply_node(const Dims& d, long long node, const T* __restrict__ K0,
                                           const T* __restrict__ x, const T* __restrict__ Ae,
                                           const VIn& vin, const T* b, T* y,
                                           const T* __restrict__ invd, T omega,
                                           const uint8_t* __restrict__ fixed,
                                           const T* __restrict__ w) {
  const long long n = d.nodes() * DIM;
  const int nnx = d.nx + 1, nny = d.ny + 1;
  int i, j, k;
  node_coords(node, nnx, nny, DIM, i, j, k);
  T acc[DIM];
  if (MODE != 3) {
    node_apply<DIM, T, FINE>(d, i, j, k, K0, x, Ae, vin, acc);
    if (w) {
      const T vl = vin(n);
#pragma unroll
      for (int c = 0; c < DIM; ++c) acc[c] = fma(w[DIM * node + c], vl, acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const long long id = DIM * node + c;
    if (!TOPO_IN(id, n)) continue;
    T out;
    if (fixed[id]) {
      out = T(0);
    } else if (MODE == 0) {
      out = acc[c];
    } else if (MODE == 1) {
      out = node_out<1, T>(acc[c], T(0), vld<COH>(b + id), T(0), omega);
    } else if (MODE == 2 || MODE == 4) {
      out = node_out<2, T>(acc[c], vin(id), vld<COH>(b + id), invd[id], omega);
    } else {
      out = node_out<3, T>(T(0), T(0), vld<COH>(b + id), invd[id], omega);
    }
    y[id] = out;
  }
}

template <int DIM, typename T, int MODE, bool FINE>
__global__ void __launch_bounds__(kThreads) k_apply(Dims d, const T* __restrict__ K0,
                                                    const T* __restrict__ x,
                                                    const T* __restrict__ Ae,
                                                    const T* __restrict__ v,
                                                    const T* __restrict__ b, T* __restrict__ y,
                                                    const T* __restrict__ invd, T omega,
                                                    const uint8_t* __restrict__ fixed,
                                                    const CgScalars* __restrict__ sc,
                                                    const T* __restrict__ w) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nodes = d.nodes();
  if (node >= nodes) return;
  const long long n = nodes * DIM;
  if constexpr (MODE == 4) {
    const VJac0<false, T> vin{b + rhs * n, invd, fixed, omega};
    apply_node<DIM, T, MODE, FINE, false>(d, node, K0, x, Ae, vin, b + rhs * n, y + rhs * n,
                                          invd, omega, fixed, w);
  } else {
    const VLoad<false, T> vin{v + rhs * n};
    apply_node<DIM, T, MODE, FINE, false>(d, node, K0, x, Ae, vin, b + rhs * n, y + rhs * n,
                                          invd, omega, fixed, w);
  }
}

// Block sum of one double per thread (deterministic tree), result valid in thread 0.
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

// The swept vector of the first two sweeps from zero on a coarse level of an IP system: VJac0 for
// the node entries and yl = omega_l b_lambda / Z_ll for the lambda entry (index n).
template <typename T>
struct VJac0Arrow {
  VJac0<false, T> u;
  long long n;
  T yl;
  __device__ __forceinline__ T operator()(long long i) const { return i == n ? yl : u(i); }
};

// Node rows of one coarse IP level over a grid-stride range of nodes; returns this thread's
// partial sum of w_i v_i (v as vin supplies it).
template <int DIM, typename T, int MODE, typename VIn>
__device__ __forceinline__ double arrow_node_rows(const Dims& d, const T* __restrict__ Ae,
                                                  const VIn& vin, const T* __restrict__ b,
                                                  T* __restrict__ y, const T* __restrict__ invd,
                                                  T omega, const uint8_t* __restrict__ fixed,
                                                  const T* __restrict__ w) {
  const long long nodes = d.nodes();
  double part = 0.0;
  for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < nodes;
       node += (long long)gridDim.x * blockDim.x) {
    apply_node<DIM, T, MODE, false, false>(d, node, nullptr, nullptr, Ae, vin, b, y, invd, omega,
                                           fixed, MODE == 3 ? nullptr : w);
    if (MODE != 3)
#pragma unroll
      for (int c = 0; c < DIM; ++c)
        part = fma((double)w[DIM * node + c], (double)vin(DIM * node + c), part);
  }
  return part;
}

// Coarse level of an IP system (the arrow matrix of Eq. (nwtr2) after Galerkin coarsening): the
// node rows of apply_node with the arrow column w, and in the same pass the lambda row
// (Z v)_lambda = w^T v_u + Z_ll v_lambda.  Each block sums w_i v_i over its nodes; the last block
// to finish adds the block sums in block order and writes y[n] per MODE, with the lambda entry's
// damping omega_l (or *wdev when the damping comes from the power iteration).  MODE 4 is the
// first two sweeps from zero in one pass (the swept vector formed on the fly by VJac0Arrow; the
// same bits as modes 3 then 2).  Grid-stride over nodes with at most kRedBlocks blocks, one
// partial sum each.
template <int DIM, typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_apply_arrow(Dims d, const T* __restrict__ Ae,
                                                          const T* __restrict__ v,
                                                          const T* __restrict__ b,
                                                          T* __restrict__ y,
                                                          const T* __restrict__ invd, T omega,
                                                          const uint8_t* __restrict__ fixed,
                                                          const CgScalars* __restrict__ sc,
                                                          const T* __restrict__ w,
                                                          const double* zll, double omega_l,
                                                          const double* wdev, double* partials,
                                                          unsigned* counter) {
  pdl_prologue();
  if (sc && sc[0].done) return;
  const long long n = d.nodes() * DIM;
  const double z = *zll, om = wdev ? *wdev : omega_l;
  T yl = T(0);
  double part;
  if constexpr (MODE == 4) {
    yl = (T)(om * (double)b[n] / z);
    const VJac0Arrow<T> vin{VJac0<false, T>{b, invd, fixed, omega}, n, yl};
    part = arrow_node_rows<DIM, T, MODE>(d, Ae, vin, b, y, invd, omega, fixed, w);
  } else {
    const VLoad<false, T> vin{v};
    part = arrow_node_rows<DIM, T, MODE>(d, Ae, vin, b, y, invd, omega, fixed, w);
  }
  __shared__ bool last;
  const double bs = block_sum(part);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  double acc = 0.0;
  for (unsigned t = threadIdx.x; t < gridDim.x; t += blockDim.x) acc += __ldcg(partials + t);
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    *counter = 0;
    double out;
    if (MODE == 3) {
      out = om * (double)b[n] / z;
    } else {
      const double vl = MODE == 4 ? (double)yl : (double)v[n];
      const double q = acc + z * vl;
      if (MODE == 0) out = q;
      else if (MODE == 1) out = (double)b[n] - q;
      else out = vl + om * ((double)b[n] - q) / z;
    }
    y[n] = (T)out;
  }
}

// 3D node-parallel operator with the right-hand sides of a node in one thread (NR of them per
// thread, grid.y chunks beyond): the element rows - x_e K0 on the finest level, K0 staged in
// shared memory; the stored Galerkin matrices below - are read once per node and applied to every
// right-hand side, where the per-right-hand-side launches read them once each.  Per right-hand
// side the arithmetic and its order are those of node_apply and apply_node (same bits).
constexpr int kApply3Threads = 128;

template <typename T, int MODE, bool FINE, int NR>
__global__ void __launch_bounds__(kApply3Threads) k_apply3_rhs(
    Dims d, const T* __restrict__ K0, const T* __restrict__ x, const T* __restrict__ Ae,
    const T* __restrict__ v, const T* __restrict__ b, T* __restrict__ y, const T* __restrict__ invd,
    T omega, const uint8_t* __restrict__ fixed, const CgScalars* __restrict__ sc, int nrhs) {
  pdl_prologue();
  constexpr int NE = 24;
  __shared__ T k0s[FINE ? NE * NE : 1];
  if (FINE) {
    for (int t = threadIdx.x; t < NE * NE; t += blockDim.x) k0s[t] = K0[t];
    __syncthreads();
  }
  const int r0 = blockIdx.y * NR;
  bool live[NR];
  bool any = false;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    live[r] = (r0 + r < nrhs) && !(sc && sc[r0 + r].done);
    any = any || live[r];
  }
  const long long nodes = d.nodes();
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nodes || !any) return;
  const long long n = nodes * 3;
  const int nnx = d.nx + 1, nny = d.ny + 1;
  const long long m = d.elems();
  int i, j, k;
  node_coords(node, nnx, nny, 3, i, j, k);
  T acc[NR][3];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r][0] = acc[r][1] = acc[r][2] = T(0);
  if (MODE != 3) {
#pragma unroll 1
    for (int s = 0; s < 8; ++s) {
      const int dx = s & 1, dy = (s >> 1) & 1, dz = s >> 2;
      const int ex = i - 1 + dx, ey = j - 1 + dy, ez = k - 1 + dz;
      if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny || ez < 0 || ez >= d.nz) continue;
      const int loc = loc_of(1 - dx, 1 - dy, 1 - dz);
      const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
      if (!TOPO_IN(e, m)) continue;
      T row[3][NE];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int q = 0; q < NE; ++q)
          row[c][q] = FINE ? k0s[(loc * 3 + c) * NE + q]
                           : ldg(Ae + (long long)((loc * 3 + c) * NE + q) * m + e);
      const T xe = FINE ? ldg(x + e) : T(0);
      long long nid[8];
#pragma unroll
      for (int a = 0; a < 8; ++a)
        nid[a] = TOPO_IDX((ex + loc_ox(a)) + (long long)nnx * ((ey + loc_oy(a)) +
                                                               (long long)nny * (ez + loc_oz(a))),
                          nodes);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (!live[r]) continue;
        const T* vr = v + (long long)(r0 + r) * n;
        T ve[NE];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) ve[a * 3 + c] = ldg(vr + 3 * nid[a] + c);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T t = T(0);
#pragma unroll
          for (int q = 0; q < NE; ++q) t = fma(row[c][q], ve[q], t);
          if (FINE) acc[r][c] = fma(xe, t, acc[r][c]);
          else acc[r][c] += t;
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (!live[r]) continue;
    const long long off = (long long)(r0 + r) * n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long id = 3 * node + c;
      if (!TOPO_IN(id, n)) continue;
      T out;
      if (fixed[id]) out = T(0);
      else if (MODE == 0) out = acc[r][c];
      else if (MODE == 1) out = node_out<1, T>(acc[r][c], T(0), ldg(b + off + id), T(0), omega);
      else if (MODE == 2)
        out = node_out<2, T>(acc[r][c], ldg(v + off + id), ldg(b + off + id), invd[id], omega);
      else out = node_out<3, T>(T(0), T(0), ldg(b + off + id), invd[id], omega);
      y[off + id] = out;
    }
  }
}

// Small coarse 3D levels: one thread per (node, element around it), NR right-hand sides per
// thread.  Each thread forms the three rows of its element's contribution for its right-hand
// sides (the multiply-add chains of k_apply3_rhs), writes them to shared memory, and one thread
// per (node, right-hand side) adds the eight elements' rows in the node's element order and
// writes the output: the arithmetic and its order are those of k_apply3_rhs (the same bits).
constexpr long long kApply3SplitNodes = 16384;
constexpr int kApply3SplitNodesPerBlock = 16;  // 128 threads

template <typename T, int MODE, int NR>
__global__ void __launch_bounds__(kApply3SplitNodesPerBlock * 8) k_apply3_split(
    Dims d, const T* __restrict__ Ae, const T* __restrict__ v, const T* __restrict__ b,
    T* __restrict__ y, const T* __restrict__ invd, T omega, const uint8_t* __restrict__ fixed,
    const CgScalars* __restrict__ sc, int nrhs) {
  pdl_prologue();
  constexpr int NE = 24;
  constexpr int NPB = kApply3SplitNodesPerBlock;
  __shared__ T part[NPB][8][NR][3];
  __shared__ bool has[NPB][8];
  const int r0 = blockIdx.y * NR;
  bool live[NR];
  bool any = false;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    live[r] = (r0 + r < nrhs) && !(sc && sc[r0 + r].done);
    any = any || live[r];
  }
  if (!any) return;  // (the same for the whole block)
  const long long nodes = d.nodes();
  const long long n = nodes * 3;
  const int nnx = d.nx + 1, nny = d.ny + 1;
  const long long m = d.elems();
  const int ln = threadIdx.x >> 3, s = threadIdx.x & 7;  // local node, element slot
  const long long node = (long long)blockIdx.x * NPB + ln;
  bool ok = false;
  if (node < nodes) {
    int i, j, k;
    node_coords(node, nnx, nny, 3, i, j, k);
    const int dx = s & 1, dy = (s >> 1) & 1, dz = s >> 2;
    const int ex = i - 1 + dx, ey = j - 1 + dy, ez = k - 1 + dz;
    ok = !(ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny || ez < 0 || ez >= d.nz);
    if (ok) {
      const int loc = loc_of(1 - dx, 1 - dy, 1 - dz);
      const long long e = TOPO_IDX(ex + (long long)d.nx * (ey + (long long)d.ny * ez), m);
      T row[3][NE];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int q = 0; q < NE; ++q) row[c][q] = ldg(Ae + (long long)((loc * 3 + c) * NE + q) * m + e);
      long long nid[8];
#pragma unroll
      for (int a = 0; a < 8; ++a)
        nid[a] = TOPO_IDX((ex + loc_ox(a)) + (long long)nnx * ((ey + loc_oy(a)) +
                                                               (long long)nny * (ez + loc_oz(a))),
                          nodes);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (!live[r]) continue;
        const T* vr = v + (long long)(r0 + r) * n;
        T ve[NE];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) ve[a * 3 + c] = ldg(vr + 3 * nid[a] + c);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T t = T(0);
#pragma unroll
          for (int q = 0; q < NE; ++q) t = fma(row[c][q], ve[q], t);
          part[ln][s][r][c] = t;
        }
      }
    }
  }
  has[ln][s] = ok;
  __syncthreads();
  // (node, right-hand side) pairs: the eight elements in slot order, as k_apply3_rhs adds them
  for (int w = threadIdx.x; w < NPB * NR; w += blockDim.x) {
    const int ln2 = w / NR, r = w % NR;
    const long long nd = (long long)blockIdx.x * NPB + ln2;
    if (nd >= nodes || !live[r]) continue;
    T acc[3] = {T(0), T(0), T(0)};
    for (int s2 = 0; s2 < 8; ++s2) {
      if (!has[ln2][s2]) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] += part[ln2][s2][r][c];
    }
    const long long off = (long long)(r0 + r) * n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long id = 3 * nd + c;
      if (!TOPO_IN(id, n)) continue;
      T out;
      if (fixed[id]) out = T(0);
      else if (MODE == 0) out = acc[c];
      else if (MODE == 1) out = node_out<1, T>(acc[c], T(0), ldg(b + off + id), T(0), omega);
      else out = node_out<2, T>(acc[c], ldg(v + off + id), ldg(b + off + id), invd[id], omega);
      y[off + id] = out;
    }
  }
}

template <typename T, int MODE, bool FINE>
void apply3_rhs_dispatch(const Dims& d, const T* K0, const T* x, const T* Ae, const T* v,
                         const T* b, T* y, const T* invd, T omega, const uint8_t* fixed, int nrhs,
                         const CgScalars* sc, cudaStream_t st) {
  const unsigned gx = blocks_for(d.nodes(), kApply3Threads);
#define TOPO_A3(NR)                                                                          \
  topo::launch(k_apply3_rhs<T, MODE, FINE, NR>, dim3(gx, (nrhs + NR - 1) / NR), kApply3Threads, \
               0, st, d, K0, x, Ae, v, b, y, invd, omega, fixed, sc, nrhs)
  // Small coarse levels (at most 16K nodes) with several right-hand sides: one thread per element
  // of a node (k_apply3_split).  With all eight elements of a node in one thread the few blocks
  // of these levels ran long serial chains of loads (the 32 x 16 x 16 and 16 x 8 x 8 levels of the
  // 128 x 64 x 64 hierarchy took about 32 us per launch; one right-hand side per thread, which
  // reads the matrices once per right-hand side, took 114-120 us).  On the 64 x 32 x 32 level
  // (70K nodes, 151 MB of matrices) the split form was slower: 101 against 73 us.
  if (!FINE && MODE != 3 && d.nodes() <= kApply3SplitNodes && nrhs >= 2) {
    const unsigned gs = blocks_for(d.nodes(), kApply3SplitNodesPerBlock);
#define TOPO_A3S(NRS)                                                                        \
  topo::launch(k_apply3_split<T, MODE, NRS>, dim3(gs, (nrhs + NRS - 1) / NRS),                \
               kApply3SplitNodesPerBlock * 8, 0, st, d, Ae, v, b, y, invd, omega, fixed, sc, nrhs)
    if (nrhs >= 5) TOPO_A3S(8);
    else TOPO_A3S(4);
#undef TOPO_A3S
    return;
  }
  if (nrhs >= 5) TOPO_A3(8);
  else if (nrhs >= 3) TOPO_A3(4);
  else if (nrhs == 2) TOPO_A3(2);
  else TOPO_A3(1);
#undef TOPO_A3
}

// First coarse level of the 2D grid without stored element matrices: the Galerkin element matrix
// of coarse element E is sum_c x_c C_c over its four children (C_c = P_c^T K0 P_c), so
// (A v)_node = sum_{E at node} sum_c x_c (C_c v_E)_row.  xf: densities of the finest level.
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_apply_l1(Dims d, const T* __restrict__ C,
                                                       const T* __restrict__ xf,
                                                       const T* __restrict__ v,
                                                       const T* __restrict__ b, T* __restrict__ y,
                                                       const T* __restrict__ invd, T omega,
                                                       const uint8_t* __restrict__ fixed,
                                                       const CgScalars* __restrict__ sc) {
  pdl_prologue();
  constexpr int NE = 8, NE2 = 64;
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nodes = d.nodes();
  if (node >= nodes) return;
  const long long n = nodes * 2;
  const int nnx = d.nx + 1;
  const int i = (int)(node % nnx), j = (int)(node / nnx);
  v += rhs * n;
  b += rhs * n;
  y += rhs * n;
  T acc[2] = {T(0), T(0)};
  const int fnx = 2 * d.nx;
  if (MODE != 3) {
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      const int dx = s & 1, dy = s >> 1;
      const int ex = i - 1 + dx, ey = j - 1 + dy;
      if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny) continue;
      const int loc = loc_of(1 - dx, 1 - dy, 0);
      T ve[NE];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const long long nid = (ex + loc_ox(a)) + (long long)nnx * (ey + loc_oy(a));
        ve[2 * a] = ldg(v + 2 * nid);
        ve[2 * a + 1] = ldg(v + 2 * nid + 1);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const long long fe = (2 * ex + (c & 1)) + (long long)fnx * (2 * ey + (c >> 1));
        const T xc = ldg(xf + fe);
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const T* row = C + c * NE2 + (loc * 2 + cc) * NE;
          T t = T(0);
#pragma unroll
          for (int q = 0; q < NE; ++q) t = fma(ldg(row + q), ve[q], t);
          acc[cc] = fma(xc, t, acc[cc]);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const long long id = 2 * node + c;
    T out;
    if (fixed[id]) out = T(0);
    else if (MODE == 0) out = acc[c];
    else if (MODE == 1) out = b[id] - acc[c];
    else if (MODE == 2) out = v[id] + omega * invd[id] * (b[id] - acc[c]);
    else out = omega * invd[id] * b[id];
    y[id] = out;
  }
}

// Threads per block of the 2D node-parallel sweeps and transfers on a level of `nodes` nodes: the
// latency-bound levels of at most 64K nodes spread their work over more SMs with 128-thread blocks
// (2048 x 1024 step: 4.514 against 4.532 ms with 256 threads; 64 threads measured in between).
static int small_level_threads(long long nodes) { return nodes <= 65536 ? 128 : kThreads; }

template <int DIM, typename T, int MODE>
void apply_dispatch(const Dims& d, const T* K0, const T* x, const T* Ae, const T* v, const T* b,
                    T* y, const T* invd, T omega, const uint8_t* fixed, int nrhs,
                    const CgScalars* sc, cudaStream_t st, const T* w) {
  dim3 grid(blocks_for(d.nodes()), nrhs);
  if constexpr (MODE <= 3) {
    if (x) {
      topo::launch(k_apply<DIM, T, MODE, true>, grid, kThreads, 0, st, d, K0, x, Ae, v, b, y, invd,
                   omega, fixed, sc, w);
      return;
    }
  }
  const int tb = DIM == 2 ? small_level_threads(d.nodes()) : kThreads;
  grid.x = blocks_for(d.nodes(), tb);
  topo::launch(k_apply<DIM, T, MODE, false>, grid, tb, 0, st, d, K0, x, Ae, v, b, y, invd,
               omega, fixed, sc, w);
}


// q = A p (FP64, finest level) with the partial sums of p^T q; the last block to finish adds the
// partials in block order and forms alpha = r^T y / p^T A p (Algorithm PCG).
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_apply_dot_fine(Dims d, const double* __restrict__ K0,
                                                             const double* __restrict__ x,
                                                             const double* __restrict__ v,
                                                             double* __restrict__ y,
                                                             const uint8_t* __restrict__ fixed,
                                                             double* partials, unsigned* counters,
                                                             CgScalars* sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc[rhs].done) return;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nodes = d.nodes();
  const long long n = nodes * DIM;
  v += rhs * n;
  y += rhs * n;
  double part = 0.0;
  if (node < nodes) {
    const int nnx = d.nx + 1, nny = d.ny + 1;
    const int i = (int)(node % nnx);
    const int j = (int)((node / nnx) % nny);
    const int k = (DIM == 3) ? (int)(node / ((long long)nnx * nny)) : 0;
    double acc[DIM];
    node_apply<DIM, double, true>(d, i, j, k, K0, x, nullptr, VLoad<false, double>{v}, acc);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const long long id = DIM * node + c;
      const double out = fixed[id] ? 0.0 : acc[c];
      y[id] = out;
      part = fma(v[id], out, part);
    }
  }
  const double bs = block_sum(part);
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
  s = block_sum(s);
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

// Restriction r_c = P^T r_f: each coarse node gathers the 3x3(x3) fine nodes around its
// coincident fine node with weights prod_d w(offset), w(0) = 1, w(+-1) = 1/2.
template <int DIM, typename T, bool COH = false>
__device__ __forceinline__ void restrict_node(const Dims& df, const Dims& dc, long long node,
                                              const T* rf, T* rc,
                                              const uint8_t* __restrict__ fixed_c) {
  const int cnx = dc.nx + 1, cny = dc.ny + 1;
  int I, J, K;
  node_coords(node, cnx, cny, DIM, I, J, K);
  const int fnx = df.nx + 1, fny = df.ny + 1;
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
  const int zlo = (DIM == 3) ? -1 : 0, zhi = (DIM == 3) ? 1 : 0;
  for (int oz = zlo; oz <= zhi; ++oz) {
    const int fk = 2 * K + oz;
    if (DIM == 3 && (fk < 0 || fk > df.nz)) continue;
    const T wz = (oz == 0) ? T(1) : T(0.5);
    for (int oy = -1; oy <= 1; ++oy) {
      const int fj = 2 * J + oy;
      if (fj < 0 || fj > df.ny) continue;
      const T wy = (oy == 0) ? wz : wz * T(0.5);
      for (int ox = -1; ox <= 1; ++ox) {
        const int fi = 2 * I + ox;
        if (fi < 0 || fi > df.nx) continue;
        const T w = (ox == 0) ? wy : wy * T(0.5);
        const long long fid = TOPO_IDX(fi + (long long)fnx * (fj + (long long)fny * (DIM == 3 ? fk : 0)),
                                       df.nodes());
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[c] = fma(w, vld<COH>(rf + DIM * fid + c), acc[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const long long id = DIM * node + c;
    if (TOPO_IN(id, dc.dofs())) rc[id] = fixed_c[id] ? T(0) : acc[c];
  }
}

template <int DIM, typename T>
__global__ void __launch_bounds__(kThreads) k_restrict(Dims df, const T* __restrict__ rf,
                                                       T* __restrict__ rc,
                                                       const uint8_t* __restrict__ fixed_c,
                                                       const CgScalars* __restrict__ sc,
                                                       int arrow) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  Dims dc{df.nx / 2, df.ny / 2, DIM == 3 ? df.nz / 2 : 1, DIM};
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (arrow && node == 0) rc[dc.dofs()] = rf[df.dofs()];
  if (node >= dc.nodes()) return;
  restrict_node<DIM, T>(df, dc, node, rf + rhs * df.dofs(), rc + rhs * dc.dofs(), fixed_c);
}

// Prolongation and correction z_f += P z_c (bilinear / trilinear interpolation).
template <int DIM, typename T, bool COH = false>
__device__ __forceinline__ void prolong_node(const Dims& df, const Dims& dc, long long node,
                                             const T* zc, T* zf,
                                             const uint8_t* __restrict__ fixed_f) {
  const int fnx = df.nx + 1, fny = df.ny + 1;
  int i, j, k;
  node_coords(node, fnx, fny, DIM, i, j, k);
  const int cnx = dc.nx + 1, cny = dc.ny + 1;
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
  const int i0 = i >> 1, i1 = (i + 1) >> 1;
  const int j0 = j >> 1, j1 = (j + 1) >> 1;
  const int k0 = k >> 1, k1 = (k + 1) >> 1;
  const T wxh = (i & 1) ? T(0.5) : T(1);
  const T wyh = (j & 1) ? T(0.5) : T(1);
  const T wzh = (DIM == 3 && (k & 1)) ? T(0.5) : T(1);
  const int nzi = (DIM == 3 && (k & 1)) ? 2 : 1;
  const int nyi = (j & 1) ? 2 : 1, nxi = (i & 1) ? 2 : 1;
  for (int a = 0; a < nzi; ++a) {
    const int K = a ? k1 : k0;
    for (int bq = 0; bq < nyi; ++bq) {
      const int J = bq ? j1 : j0;
      for (int cq = 0; cq < nxi; ++cq) {
        const int I = cq ? i1 : i0;
        const T w = wxh * wyh * wzh;
        const long long cid = TOPO_IDX(I + (long long)cnx * (J + (long long)cny * (DIM == 3 ? K : 0)),
                                       dc.nodes());
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[c] = fma(w, vld<COH>(zc + DIM * cid + c), acc[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const long long id = DIM * node + c;
    if (TOPO_IN(id, df.dofs()) && !fixed_f[id]) zf[id] = (COH ? __ldcg(zf + id) : zf[id]) + acc[c];
  }
}

// 3D prolongation and correction for NR right-hand sides per thread: the coarse indices and
// weights of a fine node are formed once and applied to every right-hand side; per right-hand
// side the multiply-adds and their order are those of prolong_node (the same bits).
template <typename T, int NR>
__global__ void __launch_bounds__(kThreads) k_prolong_add3_rhs(Dims df, const T* __restrict__ zc,
                                                               T* __restrict__ zf,
                                                               const uint8_t* __restrict__ fixed_f,
                                                               const CgScalars* __restrict__ sc,
                                                               int nrhs) {
  pdl_prologue();
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= df.nodes()) return;
  const Dims dc{df.nx / 2, df.ny / 2, df.nz / 2, 3};
  const long long nf = df.dofs(), ncd = dc.dofs();
  const int fnx = df.nx + 1, fny = df.ny + 1;
  int i, j, k;
  node_coords(node, fnx, fny, 3, i, j, k);
  const int cnx = dc.nx + 1, cny = dc.ny + 1;
  const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1, k0 = k >> 1,
            k1 = (k + 1) >> 1;
  const T wxh = (i & 1) ? T(0.5) : T(1);
  const T wyh = (j & 1) ? T(0.5) : T(1);
  const T wzh = (k & 1) ? T(0.5) : T(1);
  const T w = wxh * wyh * wzh;
  const int nzi = (k & 1) ? 2 : 1, nyi = (j & 1) ? 2 : 1, nxi = (i & 1) ? 2 : 1;
  int cid[8];  // (unrolled below: registers; grids hold < 2^31 nodes)
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int bq = 0; bq < 2; ++bq)
#pragma unroll
      for (int cq = 0; cq < 2; ++cq)
        cid[(a * 2 + bq) * 2 + cq] =
            (int)TOPO_IDX((cq ? i1 : i0) + (long long)cnx * ((bq ? j1 : j0) + (long long)cny * (a ? k1 : k0)),
                          dc.nodes());
  bool fx[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) fx[c] = fixed_f[3 * node + c] != 0;
#pragma unroll 1
  for (int r0 = 0; r0 < nrhs; r0 += NR) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int rhs = r0 + r;
      if (rhs >= nrhs || (sc && sc[rhs].done)) continue;
      const T* zr = zc + (long long)rhs * ncd;
      T* zo = zf + (long long)rhs * nf;
      T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int bq = 0; bq < 2; ++bq)
#pragma unroll
          for (int cq = 0; cq < 2; ++cq) {
            if (a >= nzi || bq >= nyi || cq >= nxi) continue;  // (the loop order of prolong_node)
            const long long q = cid[(a * 2 + bq) * 2 + cq];
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[c] = fma(w, __ldg(zr + 3 * q + c), acc[c]);
          }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long id = 3 * node + c;
        if (!fx[c] && TOPO_IN(id, nf)) zo[id] = zo[id] + acc[c];
      }
    }
  }
}

// Fine levels at or above this many nodes take every right-hand side of a node in one thread in
// the 3D prolongation (the index work once per node).
constexpr long long kBatched3Nodes = 65536;

template <int DIM, typename T>
__global__ void __launch_bounds__(kThreads) k_prolong_add(Dims df, const T* __restrict__ zc,
                                                          T* __restrict__ zf,
                                                          const uint8_t* __restrict__ fixed_f,
                                                          const CgScalars* __restrict__ sc,
                                                          int arrow) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  Dims dc{df.nx / 2, df.ny / 2, DIM == 3 ? df.nz / 2 : 1, DIM};
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (arrow && node == 0) zf[df.dofs()] += zc[dc.dofs()];
  if (node >= df.nodes()) return;
  prolong_node<DIM, T>(df, dc, node, zc + rhs * dc.dofs(), zf + rhs * df.dofs(), fixed_f);
}

// Floor of x / 2 for x >= -2 (folds to a constant for constant x).
__host__ __device__ constexpr int floor_half(int x) { return (x + 2) / 2 - 1; }

// The coarse-grid correction with the first post-smoothing sweep at one node (i, j) of a 2D level
// with stored element matrices (Algorithm MG): y = v + omega D^-1 (b - A v) with v = z + P z_c
// formed in the kernel.  The node's parities (PX, PY) = (i & 1, j & 1) are template arguments, so
// that the coarse nodes every neighbour interpolates from, and the weights, are constants.  The
// sweep reads v at the 3 x 3 neighbour nodes; each is formed once from a patch of (PX ? 2 : 3) x
// (PY ? 2 : 3) coarse nodes, with the multiply-adds in the order of prolong_node (fixed DOFs keep
// z), and the element products run as in node_apply: the bits of k_prolong_add followed by
// apply_node MODE 2.
template <typename T, int PX, int PY>
__device__ __forceinline__ void apply2_prolong_node(const Dims& d, int i, int j,
                                                    const T* __restrict__ Ae,
                                                    const T* __restrict__ z,
                                                    const T* __restrict__ zc,
                                                    const T* __restrict__ b, T* __restrict__ y,
                                                    const T* __restrict__ invd, T omega,
                                                    const uint8_t* __restrict__ fixed) {
  constexpr int NPX = PX ? 2 : 3, NPY = PY ? 2 : 3;  // the coarse patch
  const int nnx = d.nx + 1, nny = d.ny + 1;
  const long long nodes = (long long)nnx * nny, n = 2 * nodes, m = d.elems();
  const int cnx = d.nx / 2 + 1, cny = d.ny / 2 + 1;
  const long long ncn = (long long)cnx * cny;
  const int cx0 = (i >> 1) - 1 + PX, cy0 = (j >> 1) - 1 + PY;  // floor((i - 1) / 2), likewise y
  T C[NPY][NPX][2];
#pragma unroll
  for (int q = 0; q < NPY; ++q)
#pragma unroll
    for (int p = 0; p < NPX; ++p) {
      const int cx = cx0 + p, cy = cy0 + q;
      const bool in = cx >= 0 && cx < cnx && cy >= 0 && cy < cny;
      const long long cid = in ? TOPO_IDX(cx + (long long)cnx * cy, ncn) : 0;
      C[q][p][0] = in ? ldg(zc + 2 * cid) : T(0);
      C[q][p][1] = in ? ldg(zc + 2 * cid + 1) : T(0);
    }
  // the element matrix rows of the four adjacent elements (loaded before v is formed)
  T a[4][16];
  bool ok[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int dx = s & 1, dy = s >> 1;
    const int ex = i - 1 + dx, ey = j - 1 + dy;
    ok[s] = ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny;
    const int loc = loc_of(1 - dx, 1 - dy, 0);
    const long long e = ok[s] ? TOPO_IDX(ex + (long long)d.nx * ey, m) : 0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 8; ++q)
        a[s][c * 8 + q] = ldg(Ae + (long long)((loc * 2 + c) * 8 + q) * m + e);
  }
  // v at the 3 x 3 neighbours (those outside the grid are never read)
  T V[3][3][2];
#pragma unroll
  for (int dj = 0; dj < 3; ++dj)
#pragma unroll
    for (int di = 0; di < 3; ++di) {
      const int bx = PX - 1 + di, by = PY - 1 + dj;  // ii = 2 (i >> 1) + bx, likewise jj
      const int ox = bx & 1, oy = by & 1;
      const int p0 = floor_half(bx) + 1 - PX, p1 = floor_half(bx + 1) + 1 - PX;
      const int q0 = floor_half(by) + 1 - PY, q1 = floor_half(by + 1) + 1 - PY;
      const T w = (ox ? T(0.5) : T(1)) * (oy ? T(0.5) : T(1));
      const int ii = i - 1 + di, jj = j - 1 + dj;
      const bool in = ii >= 0 && ii < nnx && jj >= 0 && jj < nny;
      const long long nid = in ? TOPO_IDX(ii + (long long)nnx * jj, nodes) : 0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        T acc = fma(w, C[q0][p0][c], T(0));          // (j0, i0)
        if (ox) acc = fma(w, C[q0][p1][c], acc);      // (j0, i1)
        if (oy) {
          acc = fma(w, C[q1][p0][c], acc);            // (j1, i0)
          if (ox) acc = fma(w, C[q1][p1][c], acc);    // (j1, i1)
        }
        const long long id = 2 * nid + c;
        const T zv = in ? ldg(z + id) : T(0);
        V[dj][di][c] = (in && !fixed[id]) ? zv + acc : zv;
      }
    }
  T acc[2] = {T(0), T(0)};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (!ok[s]) continue;
    const int dx = s & 1, dy = s >> 1;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      T t = T(0);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int bq = q >> 1, cq = q & 1;
        t = fma(a[s][c * 8 + q], V[dy + loc_oy(bq)][dx + loc_ox(bq)][cq], t);
      }
      acc[c] += t;
    }
  }
  const long long node = i + (long long)nnx * j;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const long long id = 2 * node + c;
    if (!TOPO_IN(id, n)) continue;
    y[id] = fixed[id] ? T(0) : node_out<2, T>(acc[c], V[1][1][c], ldg(b + id), invd[id], omega);
  }
}

// One thread per node; blockIdx.z is the node's parity class (i & 1) + 2 (j & 1), so that every
// block runs one specialisation of apply2_prolong_node.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_apply2_prolong(Dims d, const T* __restrict__ Ae,
                                                             const T* __restrict__ z,
                                                             const T* __restrict__ zc,
                                                             const T* __restrict__ b,
                                                             T* __restrict__ y,
                                                             const T* __restrict__ invd, T omega,
                                                             const uint8_t* __restrict__ fixed,
                                                             const CgScalars* __restrict__ sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const int px = blockIdx.z & 1, py = blockIdx.z >> 1;
  const int nnx = d.nx + 1, nny = d.ny + 1;
  const int ncx = (nnx - px + 1) >> 1, ncy = (nny - py + 1) >> 1;  // nodes of the class
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= (long long)ncx * ncy) return;
  const int i = 2 * (int)(l % ncx) + px, j = 2 * (int)(l / ncx) + py;
  const long long n = 2LL * nnx * nny;
  const long long nc = 2LL * (d.nx / 2 + 1) * (d.ny / 2 + 1);
  z += rhs * n;
  b += rhs * n;
  y += rhs * n;
  zc += rhs * nc;
  switch (blockIdx.z) {
    case 0: apply2_prolong_node<T, 0, 0>(d, i, j, Ae, z, zc, b, y, invd, omega, fixed); break;
    case 1: apply2_prolong_node<T, 1, 0>(d, i, j, Ae, z, zc, b, y, invd, omega, fixed); break;
    case 2: apply2_prolong_node<T, 0, 1>(d, i, j, Ae, z, zc, b, y, invd, omega, fixed); break;
    default: apply2_prolong_node<T, 1, 1>(d, i, j, Ae, z, zc, b, y, invd, omega, fixed);
  }
}

// ---- Fused deep levels of the 2D V-cycle ----------------------------------------------------
// The levels below a few thousand nodes cost a launch per smoothing sweep, residual, restriction
// and prolongation while their work is a few microseconds of L2 traffic.  One cluster of
// kTailCluster blocks per right-hand side runs all of them, phase by phase, with the cluster
// barrier (hardware, release/acquire at cluster scope) between phases; the per-node arithmetic is
// the same device code as the unfused kernels, so the results are the same bits.  Vectors written
// within the launch are read from L2 (COH loads), never through the read-only cache.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads, 1) k_vcycle_tail(const __grid_constant__ TailArgs<T> A,
                                                                 const CgScalars* __restrict__ sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;  // the same for every block of the cluster
  const long long t0 = (long long)cluster_rank() * blockDim.x + threadIdx.x;
  const long long ts = (long long)kTailCluster * blockDim.x;
  T* res[kTailMax];
  for (int k = 0; k < A.nl - 1; ++k) {
    const Dims d = A.d[k];
    const long long n = d.dofs(), nodes = d.nodes();
    const T* b = A.b[k] + rhs * n;
    T* c = A.z[k] + rhs * n;
    T* o = A.t[k] + rhs * n;
    if (A.nu1 >= 2) {  // the first two sweeps in one phase
      const VJac0<true, T> vj{b, A.invd[k], A.fixed[k], A.omega};
      for (long long nd = t0; nd < nodes; nd += ts)
        apply_node<2, T, 4, false, true>(d, nd, nullptr, nullptr, A.Ae[k], vj, b, o, A.invd[k],
                                         A.omega, A.fixed[k], nullptr);
      cluster_barrier();
      T* tmp = c;
      c = o;
      o = tmp;
      for (int it = 2; it < A.nu1; ++it) {
        for (long long nd = t0; nd < nodes; nd += ts)
          apply_node<2, T, 2, false, true>(d, nd, nullptr, nullptr, A.Ae[k], VLoad<true, T>{c}, b,
                                           o, A.invd[k], A.omega, A.fixed[k], nullptr);
        cluster_barrier();
        tmp = c;
        c = o;
        o = tmp;
      }
    } else if (A.nu1 == 1) {
      for (long long nd = t0; nd < nodes; nd += ts)
        apply_node<2, T, 3, false, true>(d, nd, nullptr, nullptr, A.Ae[k], VLoad<true, T>{c}, b, c,
                                         A.invd[k], A.omega, A.fixed[k], nullptr);
      cluster_barrier();
    } else {
      for (long long q = t0; q < n; q += ts) c[q] = T(0);
      cluster_barrier();
    }
    for (long long nd = t0; nd < nodes; nd += ts)
      apply_node<2, T, 1, false, true>(d, nd, nullptr, nullptr, A.Ae[k], VLoad<true, T>{c}, b, o,
                                       A.invd[k], A.omega, A.fixed[k], nullptr);
    cluster_barrier();
    const Dims dc = A.d[k + 1];
    T* bc = A.b[k + 1] + rhs * dc.dofs();
    for (long long nd = t0; nd < dc.nodes(); nd += ts)
      restrict_node<2, T, true>(d, dc, nd, o, bc, A.fixed[k + 1]);
    cluster_barrier();
    res[k] = c;
  }
  {  // coarsest level: z = Ainv b, one warp per row
    const int L = A.nl - 1;
    const T* b = A.b[L] + (long long)rhs * A.nc;
    T* z = A.z[L] + (long long)rhs * A.nc;
    const int lane = threadIdx.x & 31;
    for (long long row = t0 >> 5; row < A.nc; row += ts >> 5) {
      if constexpr (sizeof(T) == 4) {
        const f2 v = dense_row_dot_df<true>(A.nc, A.AinvDF + row * A.nc, b, lane);
        if (lane == 0) z[row] = __fadd_rn(v.h, v.l);
      } else {
        const double v = dense_row_dot<true>(A.nc, A.Ainv + row * A.nc, b, lane);
        if (lane == 0) z[row] = (T)v;
      }
    }
    cluster_barrier();
    res[L] = z;
  }
  for (int k = A.nl - 2; k >= 0; --k) {
    const Dims d = A.d[k], dc = A.d[k + 1];
    const long long n = d.dofs(), nodes = d.nodes();
    const T* b = A.b[k] + rhs * n;
    T* c = res[k];
    T* zb = A.z[k] + rhs * n;
    T* o = (c == zb) ? A.t[k] + rhs * n : zb;
    // (the prolongation stays a phase of its own: a sweep that formed P z_c on the fly would do
    // so once per element entry it reads, and measured slower)
    for (long long nd = t0; nd < nodes; nd += ts)
      prolong_node<2, T, true>(d, dc, nd, res[k + 1], c, A.fixed[k]);
    cluster_barrier();
    for (int it = 0; it < A.nu2; ++it) {
      for (long long nd = t0; nd < nodes; nd += ts)
        apply_node<2, T, 2, false, true>(d, nd, nullptr, nullptr, A.Ae[k], VLoad<true, T>{c}, b, o,
                                         A.invd[k], A.omega, A.fixed[k], nullptr);
      cluster_barrier();
      T* tmp = c;
      c = o;
      o = tmp;
    }
    res[k] = c;
  }
}

// ---- Deep levels of the 2D V-cycle in one block's shared memory ----------------------------
// The cluster form above spends most of its time at the cluster barrier (a phase costs about as
// much as a launch).  From the first level of at most kTailNodes nodes down, the element matrices,
// inverse diagonals, masks and vectors of all the fused levels fit in the shared memory of one
// block (about 185 KB for the 32 x 16, 16 x 8 and 8 x 4 levels in FP32).  One block per
// right-hand side copies them in once per V-cycle and runs every phase on shared memory with
// __syncthreads between phases; only the coarsest inverse is read from global memory.  The
// per-node arithmetic and its order are those of the unfused kernels (node_apply's coarse 2D
// branch, node_out, restrict_node, prolong_node, dense_row_dot), so the bits are the same.
template <typename T>
struct SmVec {
  const T* v;
  __device__ __forceinline__ T operator()(long long i) const { return v[i]; }
};
template <typename T>
struct SmJac0 {  // omega invd b, as VJac0 forms it
  const T* b;
  const T* invd;
  const uint8_t* fixed;
  T omega;
  __device__ __forceinline__ T operator()(long long i) const {
    return fixed[i] ? T(0) : mul_rn(mul_rn(omega, invd[i]), b[i]);
  }
};

// Bulk copies global -> shared by the tensor memory accelerator, completing on an mbarrier.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// Asynchronous 4- or 8-byte global -> shared copy (completes at cp.async.wait_all).
template <int BYTES>
__device__ __forceinline__ void cp_async_g2s(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src),
               "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes,
                                         unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// Waits for phase 0 of the barrier for at most limit_ns of the global timer (each poll may
// suspend the thread for up to 1 us); false if it gave up.  limit_ns = 0 gives up at once without
// polling (topo_set_wait_limit_ns: the timeout path made to run, for tests).
constexpr unsigned long long kBulkWaitNs = 1000000000ull;
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait0(unsigned bar,
                                           unsigned long long limit_ns = kBulkWaitNs) {
  if (limit_ns == 0) return false;
  const unsigned long long t0 = global_ns();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, 1000;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

template <int MODE, typename T, typename VIn>
__device__ __forceinline__ void sm_apply(const Dims& d, int node, const T* M, const VIn& vin,
                                         const T* B, const T* D, const uint8_t* F, T* Y,
                                         T omega) {
  const int nnx = d.nx + 1;
  const int m = d.nx * d.ny;
  const int i = node % nnx, j = node / nnx;
  T acc[2] = {T(0), T(0)};
  if (MODE != 3) {
    T a[4][16], ve[4][8];
    bool ok[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int dx = s & 1, dy = s >> 1;
      const int ex = i - 1 + dx, ey = j - 1 + dy;
      ok[s] = ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny;
      const int loc = loc_of(1 - dx, 1 - dy, 0);
      const int e = ok[s] ? ex + d.nx * ey : 0;
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int q = 0; q < 8; ++q) a[s][c * 8 + q] = M[((loc * 2 + c) * 8 + q) * m + e];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int nid = ok[s] ? (ex + loc_ox(b)) + nnx * (ey + loc_oy(b)) : 0;
        ve[s][2 * b] = vin(2 * nid);
        ve[s][2 * b + 1] = vin(2 * nid + 1);
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (!ok[s]) continue;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        T t = T(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) t = fma(a[s][c * 8 + q], ve[s][q], t);
        acc[c] += t;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int id = 2 * node + c;
    T out;
    if (F[id]) out = T(0);
    else if (MODE == 1) out = node_out<1, T>(acc[c], T(0), B[id], T(0), omega);
    else if (MODE == 2 || MODE == 4) out = node_out<2, T>(acc[c], vin(id), B[id], D[id], omega);
    else out = node_out<3, T>(T(0), T(0), B[id], D[id], omega);
    Y[id] = out;
  }
}

// The node rows of sm_apply with the element matrices element-major (kAemStride entries per
// element, rows loc*2 and loc*2+1 contiguous: four 16-byte loads per element in FP32) and the
// 3 x 3 node neighbourhood loaded once (18 values instead of 32).  The values, the FMA chains and
// their order are those of sm_apply (the same bits).
// (A coarsest system above kTail1MaxNc DOFs keeps the cluster form: its dense solve, nc^2 FP64
// multiply-adds, is FP64-bound on one SM - 306 DOFs took 78 us in one block.)
constexpr int kTail1MaxNc = 128;

template <typename T>
__device__ __forceinline__ void load16(const T* p, T out[16]) {
  if constexpr (sizeof(T) == 4) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 w = q[u];
      out[4 * u] = w.x;
      out[4 * u + 1] = w.y;
      out[4 * u + 2] = w.z;
      out[4 * u + 3] = w.w;
    }
  } else {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double2 w = q[u];
      out[2 * u] = w.x;
      out[2 * u + 1] = w.y;
    }
  }
}

template <int MODE, typename T, typename VIn>
__device__ __forceinline__ void sm_apply_em(const Dims& d, int node, const T* Me, const VIn& vin,
                                            const T* B, const T* D, const uint8_t* F, T* Y,
                                            T omega) {
  const int nnx = d.nx + 1;
  const int i = node % nnx, j = node / nnx;
  T acc[2] = {T(0), T(0)};
  T own[2] = {T(0), T(0)};
  if (MODE != 3) {
    T nv[3][3][2];  // nodes (i - 1 + a, j - 1 + b) at nv[b][a]; outside the grid: unused zeros
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int ni = i - 1 + a, nj = j - 1 + b;
        const bool ok = ni >= 0 && ni <= d.nx && nj >= 0 && nj <= d.ny;
        const int nid = ok ? ni + nnx * nj : 0;
        nv[b][a][0] = ok ? vin(2 * nid) : T(0);
        nv[b][a][1] = ok ? vin(2 * nid + 1) : T(0);
      }
    own[0] = nv[1][1][0];
    own[1] = nv[1][1][1];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int dx = s & 1, dy = s >> 1;
      const int ex = i - 1 + dx, ey = j - 1 + dy;
      if (!(ex >= 0 && ex < d.nx && ey >= 0 && ey < d.ny)) continue;
      const int loc = loc_of(1 - dx, 1 - dy, 0);
      T a[16];
      load16(Me + (ex + d.nx * ey) * kAemStride + loc * 16, a);
      T ve[8];
#pragma unroll
      for (int bq = 0; bq < 4; ++bq) {
        ve[2 * bq] = nv[dy + loc_oy(bq)][dx + loc_ox(bq)][0];
        ve[2 * bq + 1] = nv[dy + loc_oy(bq)][dx + loc_ox(bq)][1];
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        T t = T(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) t = fma(a[c * 8 + q], ve[q], t);
        acc[c] += t;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int id = 2 * node + c;
    T out;
    if (F[id]) out = T(0);
    else if (MODE == 1) out = node_out<1, T>(acc[c], T(0), B[id], T(0), omega);
    else if (MODE == 2 || MODE == 4) out = node_out<2, T>(acc[c], own[c], B[id], D[id], omega);
    else out = node_out<3, T>(T(0), T(0), B[id], D[id], omega);
    Y[id] = out;
  }
}

template <typename T>
__device__ __forceinline__ void sm_restrict(const Dims& df, const Dims& dc, int node, const T* rf,
                                            T* rc, const uint8_t* fixed_c) {
  const int cnx = dc.nx + 1;
  const int I = node % cnx, J = node / cnx;
  T acc[2] = {T(0), T(0)};
  for (int oy = -1; oy <= 1; ++oy) {
    const int fj = 2 * J + oy;
    if (fj < 0 || fj > df.ny) continue;
    const T wy = (oy == 0) ? T(1) : T(1) * T(0.5);
    for (int ox = -1; ox <= 1; ++ox) {
      const int fi = 2 * I + ox;
      if (fi < 0 || fi > df.nx) continue;
      const T w = (ox == 0) ? wy : wy * T(0.5);
      const int fid = fi + (df.nx + 1) * fj;
#pragma unroll
      for (int c = 0; c < 2; ++c) acc[c] = fma(w, rf[2 * fid + c], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) rc[2 * node + c] = fixed_c[2 * node + c] ? T(0) : acc[c];
}

template <typename T>
__device__ __forceinline__ void sm_prolong(const Dims& df, const Dims& dc, int node, const T* zc,
                                           T* zf, const uint8_t* fixed_f) {
  const int fnx = df.nx + 1, cnx = dc.nx + 1;
  const int i = node % fnx, j = node / fnx;
  T acc[2] = {T(0), T(0)};
  const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1;
  const T wxh = (i & 1) ? T(0.5) : T(1);
  const T wyh = (j & 1) ? T(0.5) : T(1);
  const T wzh = T(1);
  const int nyi = (j & 1) ? 2 : 1, nxi = (i & 1) ? 2 : 1;
  for (int bq = 0; bq < nyi; ++bq) {
    const int J = bq ? j1 : j0;
    for (int cq = 0; cq < nxi; ++cq) {
      const int I = cq ? i1 : i0;
      const T w = wxh * wyh * wzh;
      const int cid = I + cnx * J;
#pragma unroll
      for (int c = 0; c < 2; ++c) acc[c] = fma(w, zc[2 * cid + c], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int id = 2 * node + c;
    if (!fixed_f[id]) zf[id] = zf[id] + acc[c];
  }
}

// (FP64: half the threads, so that the 96 values a node gathers stay in registers)
template <typename T>
constexpr int tail1_threads() { return sizeof(T) == 8 ? kTail1Threads / 2 : kTail1Threads; }

template <typename T>
__global__ void __launch_bounds__(tail1_threads<T>(), 1)
    k_vcycle_tail1(const __grid_constant__ TailArgs<T> A, const CgScalars* __restrict__ sc) {
  pdl_prologue();
  const int rhs = blockIdx.x;
  if (sc && sc[rhs].done) return;
  extern __shared__ float4 tail1_raw[];
  char* sm = reinterpret_cast<char*>(tail1_raw);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int L = A.nl - 1;  // the coarsest, relative
  // the coarsest inverse is read once per cycle from global memory: bring it to L2 now
  const char* ainv = sizeof(T) == 4 ? reinterpret_cast<const char*>(A.AinvDF)
                                    : reinterpret_cast<const char*>(A.Ainv);  // (8 B per entry)
  for (long long q = (long long)tid * 128; q < (long long)A.nc * A.nc * 8; q += (long long)nt * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ainv + q));
  // every fused level's matrices by bulk copies on one barrier, the inverse diagonals, masks and
  // the first level's b by plain loads meanwhile
  uint64_t* bar_p = reinterpret_cast<uint64_t*>(sm + A.off_bar);
  const unsigned bar = smem_addr(bar_p);
  if (tid == 0) {
    mbar_init(bar);
    unsigned bytes = 0;
    for (int k = 0; k < L; ++k) bytes += (unsigned)(kAemStride * A.d[k].elems() * sizeof(T));
    mbar_expect_tx(bar, bytes);
    for (int k = 0; k < L; ++k)
      bulk_g2s(smem_addr(sm + A.off_m[k]), A.Aem[k],
               (unsigned)(kAemStride * A.d[k].elems() * sizeof(T)),
               bar);
  }
  // (asynchronous copies, all in flight together: plain loads level by level took 4 us)
#pragma unroll 1
  for (int k = 0; k < A.nl; ++k) {
    const int n = (int)A.d[k].dofs();
    uint8_t* F = reinterpret_cast<uint8_t*>(sm + A.off_f[k]);
    const int nw4 = n >> 2;  // the mask in 4-byte words, the last n % 4 bytes plainly
    for (int i = tid; i < nw4; i += nt) cp_async_g2s<4>(F + 4 * i, A.fixed[k] + 4 * i);
    for (int i = 4 * nw4 + tid; i < n; i += nt) F[i] = A.fixed[k][i];
    if (k == L) continue;
    T* D = reinterpret_cast<T*>(sm + A.off_d[k]);
    for (int i = tid; i < n; i += nt) cp_async_g2s<sizeof(T)>(D + i, A.invd[k] + i);
    if (k == 0) {
      T* B = reinterpret_cast<T*>(sm + A.off_b[k]);
      const T* b = A.b[0] + (long long)rhs * n;
      for (int i = tid; i < n; i += nt) cp_async_g2s<sizeof(T)>(B + i, b + i);
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();  // (the barrier is initialised before anyone polls it)
  // every thread polls; the block decides together, so that all or none continue
  if (!__syncthreads_and(mbar_wait0(bar, A.wait_ns) ? 1 : 0)) {
    // the copies did not land in time: give them a second bounded wait (the full bound) before
    // the block's shared memory is released, and stop this right-hand side's CG with a timeout
    if (tid == 0) {
      mbar_wait0(bar, kBulkWaitNs);
      if (sc) {
        CgScalars* w = const_cast<CgScalars*>(sc) + rhs;
        w->status = TOPO_E_TIMEOUT;
        w->done = 1;
      }
    }
    return;
  }
  T* res[kTailMax];
#pragma unroll 1
  for (int k = 0; k < L; ++k) {
    const Dims d = A.d[k];
    const int n = (int)d.dofs(), nodes = (int)d.nodes();
    const T* M = reinterpret_cast<const T*>(sm + A.off_m[k]);
    const T* B = reinterpret_cast<const T*>(sm + A.off_b[k]);
    const T* D = reinterpret_cast<const T*>(sm + A.off_d[k]);
    const uint8_t* F = reinterpret_cast<const uint8_t*>(sm + A.off_f[k]);
    T* c = reinterpret_cast<T*>(sm + A.off_z[k]);
    T* o = reinterpret_cast<T*>(sm + A.off_t[k]);
    if (A.nu1 >= 2) {  // the first two sweeps in one phase
      for (int nd = tid; nd < nodes; nd += nt)
        sm_apply_em<4>(d, nd, M, SmJac0<T>{B, D, F, A.omega}, B, D, F, o, A.omega);
      __syncthreads();
      T* tmp = c;
      c = o;
      o = tmp;
      for (int it = 2; it < A.nu1; ++it) {
        for (int nd = tid; nd < nodes; nd += nt)
          sm_apply_em<2>(d, nd, M, SmVec<T>{c}, B, D, F, o, A.omega);
        __syncthreads();
        tmp = c;
        c = o;
        o = tmp;
      }
    } else if (A.nu1 == 1) {
      for (int nd = tid; nd < nodes; nd += nt)
        sm_apply_em<3>(d, nd, M, SmVec<T>{c}, B, D, F, c, A.omega);
      __syncthreads();
    } else {
      for (int q = tid; q < n; q += nt) c[q] = T(0);
      __syncthreads();
    }
    for (int nd = tid; nd < nodes; nd += nt)
      sm_apply_em<1>(d, nd, M, SmVec<T>{c}, B, D, F, o, A.omega);
    __syncthreads();
    const Dims dc = A.d[k + 1];
    T* bc = reinterpret_cast<T*>(sm + A.off_b[k + 1]);
    const uint8_t* Fc = reinterpret_cast<const uint8_t*>(sm + A.off_f[k + 1]);
    for (int nd = tid; nd < (int)dc.nodes(); nd += nt) sm_restrict<T>(d, dc, nd, o, bc, Fc);
    __syncthreads();
    res[k] = c;
  }
  {  // coarsest level: z = Ainv b, one warp per row, the sums of dense_row_dot_df (FP32 vectors)
     // or dense_row_dot (FP64) in their order (the same bits); kRows rows per warp with every
     // load of a round issued before the first product
    const T* b = reinterpret_cast<const T*>(sm + A.off_b[L]);
    T* z = reinterpret_cast<T*>(sm + A.off_z[L]);
    const int lane = tid & 31, nw = nt >> 5;
    constexpr int kRows = 3, kPer = kTail1MaxNc / 32;
    const int nc = A.nc;
    T bv[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int k = lane + 32 * j;
      bv[j] = k < nc ? b[k] : T(0);
    }
    for (int row0 = tid >> 5; row0 < nc; row0 += kRows * nw) {
      if constexpr (sizeof(T) == 4) {
        float2 a[kRows][kPer];
#pragma unroll
        for (int r = 0; r < kRows; ++r)
#pragma unroll
          for (int j = 0; j < kPer; ++j) {
            const int row = row0 + r * nw, k = lane + 32 * j;
            a[r][j] = (row < nc && k < nc) ? __ldg(A.AinvDF + (long long)row * nc + k)
                                           : make_float2(0.f, 0.f);
          }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
          const int row = row0 + r * nw;
          f2 sum = {0.0f, 0.0f};
#pragma unroll
          for (int j = 0; j < kPer; ++j)
            if (lane + 32 * j < nc) sum = df_fma_f(f2{a[r][j].x, a[r][j].y}, bv[j], sum);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
            sum = df_add(sum, f2{__shfl_xor_sync(0xffffffffu, sum.h, o),
                                 __shfl_xor_sync(0xffffffffu, sum.l, o)});
          if (lane == 0 && row < nc) z[row] = __fadd_rn(sum.h, sum.l);
        }
      } else {
        double a[kRows][kPer];
#pragma unroll
        for (int r = 0; r < kRows; ++r)
#pragma unroll
          for (int j = 0; j < kPer; ++j) {
            const int row = row0 + r * nw, k = lane + 32 * j;
            a[r][j] = (row < nc && k < nc) ? __ldg(A.Ainv + (long long)row * nc + k) : 0.0;
          }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
          const int row = row0 + r * nw;
          double sum = 0.0;
#pragma unroll
          for (int j = 0; j < kPer; ++j)
            if (lane + 32 * j < nc) sum = fma(a[r][j], double_of(bv[j]), sum);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          if (lane == 0 && row < nc) z[row] = (T)sum;
        }
      }
    }
    __syncthreads();
    res[L] = z;
  }
#pragma unroll 1
  for (int k = L - 1; k >= 0; --k) {
    const Dims d = A.d[k], dc = A.d[k + 1];
    const int nodes = (int)d.nodes();
    const T* M = reinterpret_cast<const T*>(sm + A.off_m[k]);
    const T* B = reinterpret_cast<const T*>(sm + A.off_b[k]);
    const T* D = reinterpret_cast<const T*>(sm + A.off_d[k]);
    const uint8_t* F = reinterpret_cast<const uint8_t*>(sm + A.off_f[k]);
    T* zs = reinterpret_cast<T*>(sm + A.off_z[k]);
    T* c = res[k];
    T* o = (c == zs) ? reinterpret_cast<T*>(sm + A.off_t[k]) : zs;
    for (int nd = tid; nd < nodes; nd += nt) sm_prolong<T>(d, dc, nd, res[k + 1], c, F);
    __syncthreads();
    for (int it = 0; it < A.nu2; ++it) {
      for (int nd = tid; nd < nodes; nd += nt)
        sm_apply_em<2>(d, nd, M, SmVec<T>{c}, B, D, F, o, A.omega);
      __syncthreads();
      T* tmp = c;
      c = o;
      o = tmp;
    }
    res[k] = c;
  }
  const int n0 = (int)A.d[0].dofs();
  T* out = A.z[0] + (long long)rhs * n0;
  for (int i = tid; i < n0; i += nt) out[i] = res[0][i];
}

// 1 / diag(A) per DOF (1 on fixed DOFs).
template <int DIM>
__global__ void k_inv_diag(Dims d, const double* __restrict__ K0, const double* __restrict__ x,
                           const double* __restrict__ Ae, const uint8_t* __restrict__ fixed,
                           double* __restrict__ invd) {
  pdl_prologue();
  constexpr int NN = Elem<DIM>::NN, NE = Elem<DIM>::NE;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= d.nodes()) return;
  const int nnx = d.nx + 1, nny = d.ny + 1;
  const int i = (int)(node % nnx), j = (int)((node / nnx) % nny);
  const int k = (DIM == 3) ? (int)(node / ((long long)nnx * nny)) : 0;
  double acc[DIM] = {};
  for (int s = 0; s < NN; ++s) {
    const int dx = s & 1, dy = (s >> 1) & 1, dz = (DIM == 3) ? (s >> 2) : 0;
    const int ex = i - 1 + dx, ey = j - 1 + dy, ez = (DIM == 3) ? k - 1 + dz : 0;
    if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny) continue;
    if (DIM == 3 && (ez < 0 || ez >= d.nz)) continue;
    const int loc = loc_of(1 - dx, 1 - dy, DIM == 3 ? 1 - dz : 0);
    const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
    for (int c = 0; c < DIM; ++c) {
      const int r = loc * DIM + c;
      acc[c] += x ? x[e] * K0[r * NE + r] : Ae[(long long)(r * NE + r) * d.elems() + e];
    }
  }
  for (int c = 0; c < DIM; ++c) {
    const long long id = DIM * node + c;
    invd[id] = (fixed[id] || !(acc[c] > 0.0)) ? 1.0 : 1.0 / acc[c];
  }
}

// FP32 variant for coarse levels whose element matrices are stored in FP32 only.
template <int DIM>
__global__ void k_inv_diag32(Dims d, const float* __restrict__ Ae,
                             const uint8_t* __restrict__ fixed, float* __restrict__ invd) {
  pdl_prologue();
  constexpr int NN = Elem<DIM>::NN, NE = Elem<DIM>::NE;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= d.nodes()) return;
  const int nnx = d.nx + 1, nny = d.ny + 1;
  const int i = (int)(node % nnx), j = (int)((node / nnx) % nny);
  const int k = (DIM == 3) ? (int)(node / ((long long)nnx * nny)) : 0;
  float acc[DIM] = {};
  for (int s = 0; s < NN; ++s) {
    const int dx = s & 1, dy = (s >> 1) & 1, dz = (DIM == 3) ? (s >> 2) : 0;
    const int ex = i - 1 + dx, ey = j - 1 + dy, ez = (DIM == 3) ? k - 1 + dz : 0;
    if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny) continue;
    if (DIM == 3 && (ez < 0 || ez >= d.nz)) continue;
    const int loc = loc_of(1 - dx, 1 - dy, DIM == 3 ? 1 - dz : 0);
    const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
    for (int c = 0; c < DIM; ++c) {
      const int r = loc * DIM + c;
      acc[c] += Ae[(long long)(r * NE + r) * d.elems() + e];
    }
  }
  for (int c = 0; c < DIM; ++c) {
    const long long id = DIM * node + c;
    invd[id] = (fixed[id] || !(acc[c] > 0.0f)) ? 1.0f : 1.0f / acc[c];
  }
}

// E_e = scale * lam_e^T K0 u_e (lam = u gives the element energy u_e^T K0 u_e).
template <int DIM>
__global__ void k_element_energy(Dims d, const double* __restrict__ K0,
                                 const double* __restrict__ u, const double* __restrict__ lam,
                                 double* __restrict__ out, double scale) {
  pdl_prologue();
  constexpr int NN = Elem<DIM>::NN, NE = Elem<DIM>::NE;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.elems()) return;
  const int ex = (int)(e % d.nx), ey = (int)((e / d.nx) % d.ny);
  const int ez = (DIM == 3) ? (int)(e / ((long long)d.nx * d.ny)) : 0;
  const int nnx = d.nx + 1, nny = d.ny + 1;
  double ue[NE], le[NE];
#pragma unroll
  for (int a = 0; a < NN; ++a) {
    const long long nid = (ex + loc_ox(a)) + (long long)nnx * ((ey + loc_oy(a)) +
                                                               (long long)nny * (ez + loc_oz(a)));
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      ue[a * DIM + c] = u[DIM * nid + c];
      le[a * DIM + c] = lam[DIM * nid + c];
    }
  }
  double s = 0.0;
  for (int r = 0; r < NE; ++r) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < NE; ++q) t = fma(__ldg(K0 + r * NE + q), ue[q], t);
    s = fma(le[r], t, s);
  }
  out[e] = scale * s;
}

// flag = 1 if any x_i is not finite or not > 0 (x_i > 0 is false for NaN).
__global__ void k_check_positive(const double* __restrict__ x, long long m, int* flag) {
  pdl_prologue();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    const double v = x[i];
    if (!(v > 0.0) || !isfinite(v)) *flag = 1;
  }
}

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, long long n) {
  pdl_prologue();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, long long n) {
  pdl_prologue();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

}  // namespace

template <typename T>
cudaError_t launch_apply(const Dims& d, int mode, const T* K0, const T* x, const T* Ae, const T* v,
                         const T* b, T* y, const T* invd, T omega, const uint8_t* fixed, int nrhs,
                         const CgScalars* sc, cudaStream_t st, const T* w) {
#define TOPO_APPLY_CASE(DIM)                                                                     \
  switch (mode) {                                                                                \
    case 0:                                                                                      \
      apply_dispatch<DIM, T, 0>(d, K0, x, Ae, v, b, y, invd, omega, fixed, nrhs, sc, st, w); \
      break;                                                                                     \
    case 1:                                                                                      \
      apply_dispatch<DIM, T, 1>(d, K0, x, Ae, v, b, y, invd, omega, fixed, nrhs, sc, st, w); \
      break;                                                                                     \
    case 2:                                                                                      \
      apply_dispatch<DIM, T, 2>(d, K0, x, Ae, v, b, y, invd, omega, fixed, nrhs, sc, st, w); \
      break;                                                                                     \
    default:                                                                                     \
      apply_dispatch<DIM, T, 3>(d, K0, x, Ae, v, b, y, invd, omega, fixed, nrhs, sc, st, w); \
  }
  if (d.dim == 2) {
    if (mode == 4 && !x && !w) {
      apply_dispatch<2, T, 4>(d, K0, x, Ae, v, b, y, invd, omega, fixed, nrhs, sc, st, w);
    } else if (mode >= 4) {
      return cudaErrorInvalidValue;  // the fused mode: 2D stored element matrices, no arrow
    } else {
      TOPO_APPLY_CASE(2)
    }
  } else {
    if (mode >= 4) return cudaErrorInvalidValue;
    if (!w) {  // every right-hand side of a node in one thread
#define TOPO_A3_MODE(MODE)                                                                    \
  if (x) apply3_rhs_dispatch<T, MODE, true>(d, K0, x, Ae, v, b, y, invd, omega, fixed, nrhs, sc, st); \
  else apply3_rhs_dispatch<T, MODE, false>(d, K0, x, Ae, v, b, y, invd, omega, fixed, nrhs, sc, st)
      switch (mode) {
        case 0: TOPO_A3_MODE(0); break;
        case 1: TOPO_A3_MODE(1); break;
        case 2: TOPO_A3_MODE(2); break;
        default: TOPO_A3_MODE(3);
      }
#undef TOPO_A3_MODE
    } else {
      TOPO_APPLY_CASE(3)
    }
  }
#undef TOPO_APPLY_CASE
  return cudaGetLastError();
}

template cudaError_t launch_apply<double>(const Dims&, int, const double*, const double*,
                                          const double*, const double*, const double*, double*,
                                          const double*, double, const uint8_t*, int,
                                          const CgScalars*, cudaStream_t, const double*);
template cudaError_t launch_apply<float>(const Dims&, int, const float*, const float*, const float*,
                                         const float*, const float*, float*, const float*, float,
                                         const uint8_t*, int, const CgScalars*, cudaStream_t,
                                         const float*);

template <typename T>
cudaError_t launch_apply_arrow(const Dims& d, int mode, const T* Ae, const T* v, const T* b, T* y,
                               const T* invd, T omega, const uint8_t* fixed, const T* w,
                               const double* zll, double omega_l, const double* wdev,
                               double* partials, unsigned* counter, const CgScalars* sc,
                               cudaStream_t st) {
  const long long nb = blocks_for(d.nodes());
  const unsigned grid = (unsigned)(nb < kRedBlocks ? nb : kRedBlocks);
#define TOPO_ARROW(DIM, MODE)                                                                  \
  topo::launch(k_apply_arrow<DIM, T, MODE>, grid, kThreads, 0, st, d, Ae, v, b, y, invd, omega, \
               fixed, sc, w, zll, omega_l, wdev, partials, counter)
#define TOPO_ARROW_MODES(DIM)          \
  switch (mode) {                      \
    case 0: TOPO_ARROW(DIM, 0); break; \
    case 1: TOPO_ARROW(DIM, 1); break; \
    case 2: TOPO_ARROW(DIM, 2); break; \
    case 3: TOPO_ARROW(DIM, 3); break; \
    default: return cudaErrorInvalidValue; \
  }
  if (d.dim == 2 && mode == 4) {
    TOPO_ARROW(2, 4);
  } else if (d.dim == 2) {
    TOPO_ARROW_MODES(2)
  } else {
    TOPO_ARROW_MODES(3)
  }
#undef TOPO_ARROW_MODES
#undef TOPO_ARROW
  return cudaGetLastError();
}
template cudaError_t launch_apply_arrow<double>(const Dims&, int, const double*, const double*,
                                                const double*, double*, const double*, double,
                                                const uint8_t*, const double*, const double*,
                                                double, const double*, double*, unsigned*,
                                                const CgScalars*, cudaStream_t);
template cudaError_t launch_apply_arrow<float>(const Dims&, int, const float*, const float*,
                                               const float*, float*, const float*, float,
                                               const uint8_t*, const float*, const double*, double,
                                               const double*, double*, unsigned*, const CgScalars*,
                                               cudaStream_t);

template <typename T>
cudaError_t launch_apply_l1(const Dims& d, int mode, const T* C, const T* xf, const T* v,
                            const T* b, T* y, const T* invd, T omega, const uint8_t* fixed,
                            int nrhs, const CgScalars* sc, cudaStream_t st) {
  dim3 grid(blocks_for(d.nodes()), nrhs);
  switch (mode) {
    case 0:
      topo::launch(k_apply_l1<T, 0>, grid, kThreads, 0, st, d, C, xf, v, b, y, invd, omega, fixed, sc);
      break;
    case 1:
      topo::launch(k_apply_l1<T, 1>, grid, kThreads, 0, st, d, C, xf, v, b, y, invd, omega, fixed, sc);
      break;
    case 2:
      topo::launch(k_apply_l1<T, 2>, grid, kThreads, 0, st, d, C, xf, v, b, y, invd, omega, fixed, sc);
      break;
    default:
      topo::launch(k_apply_l1<T, 3>, grid, kThreads, 0, st, d, C, xf, v, b, y, invd, omega, fixed, sc);
  }
  return cudaGetLastError();
}
template cudaError_t launch_apply_l1<float>(const Dims&, int, const float*, const float*,
                                            const float*, const float*, float*, const float*,
                                            float, const uint8_t*, int, const CgScalars*,
                                            cudaStream_t);
template cudaError_t launch_apply_l1<double>(const Dims&, int, const double*, const double*,
                                             const double*, const double*, double*,
                                             const double*, double, const uint8_t*, int,
                                             const CgScalars*, cudaStream_t);

cudaError_t launch_apply_dot_fine(const Dims& d, const double* K0, const double* x, const double* v,
                                  double* y, const uint8_t* fixed, int nrhs, double* partials,
                                  unsigned* counters, CgScalars* sc, cudaStream_t st) {
  dim3 grid(blocks_for(d.nodes()), nrhs);
  if (d.dim == 2)
    topo::launch(k_apply_dot_fine<2>, grid, kThreads, 0, st, d, K0, x, v, y, fixed, partials, counters, sc);
  else
    topo::launch(k_apply_dot_fine<3>, grid, kThreads, 0, st, d, K0, x, v, y, fixed, partials, counters, sc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const Dims& fine, const T* rf, T* rc, const uint8_t* fixed_c, int nrhs,
                            const CgScalars* sc, cudaStream_t st, int arrow) {
  Dims dc{fine.nx / 2, fine.ny / 2, fine.dim == 3 ? fine.nz / 2 : 1, fine.dim};
  dim3 grid(blocks_for(dc.nodes()), nrhs);
  if (fine.dim == 2) {
    const int tb = small_level_threads(fine.nodes());
    grid.x = blocks_for(dc.nodes(), tb);
    topo::launch(k_restrict<2, T>, grid, tb, 0, st, fine, rf, rc, fixed_c, sc, arrow);
  } else  // (one thread per right-hand side: a form with every right-hand side of a coarse node in
        // one thread measured 30 against 19 us on the 1.6M-DOF level with 8 right-hand sides)
    topo::launch(k_restrict<3, T>, grid, kThreads, 0, st, fine, rf, rc, fixed_c, sc, arrow);
  return cudaGetLastError();
}
template cudaError_t launch_restrict<double>(const Dims&, const double*, double*, const uint8_t*,
                                             int, const CgScalars*, cudaStream_t, int);
template cudaError_t launch_restrict<float>(const Dims&, const float*, float*, const uint8_t*, int,
                                            const CgScalars*, cudaStream_t, int);

template <typename T>
cudaError_t launch_prolong_add(const Dims& fine, const T* zc, T* zf, const uint8_t* fixed_f,
                               int nrhs, const CgScalars* sc, cudaStream_t st, int arrow) {
  dim3 grid(blocks_for(fine.nodes()), nrhs);
  if (fine.dim == 2) {
    const int tb = small_level_threads(fine.nodes());
    grid.x = blocks_for(fine.nodes(), tb);
    topo::launch(k_prolong_add<2, T>, grid, tb, 0, st, fine, zc, zf, fixed_f, sc, arrow);
  }
  else if (nrhs >= 2 && !arrow && fine.nodes() >= kBatched3Nodes)
    // (every right-hand side of a node in one thread: 71 -> 30 us on the 1.6M-DOF level with 8
    // right-hand sides; on levels of a few thousand nodes one thread per right-hand side is faster)
    topo::launch(k_prolong_add3_rhs<T, 1>, dim3(blocks_for(fine.nodes())), kThreads, 0, st, fine,
                 zc, zf, fixed_f, sc, nrhs);
  else
    topo::launch(k_prolong_add<3, T>, grid, kThreads, 0, st, fine, zc, zf, fixed_f, sc, arrow);
  return cudaGetLastError();
}
template cudaError_t launch_prolong_add<double>(const Dims&, const double*, double*,
                                                const uint8_t*, int, const CgScalars*,
                                                cudaStream_t, int);
template cudaError_t launch_prolong_add<float>(const Dims&, const float*, float*, const uint8_t*,
                                               int, const CgScalars*, cudaStream_t, int);

template <typename T>
cudaError_t launch_apply2_prolong(const Dims& d, const T* Ae, const T* z, const T* zc, const T* b,
                                  T* y, const T* invd, T omega, const uint8_t* fixed, int nrhs,
                                  const CgScalars* sc, cudaStream_t st) {
  if (d.dim != 2 || (d.nx & 1) || (d.ny & 1) || !Ae) return cudaErrorInvalidValue;
  // (the largest parity class: the even nodes, (nx / 2 + 1) (ny / 2 + 1))
  const int tb = small_level_threads(d.nodes());
  dim3 grid(blocks_for((long long)(d.nx / 2 + 1) * (d.ny / 2 + 1), tb), nrhs, 4);
  topo::launch(k_apply2_prolong<T>, grid, tb, 0, st, d, Ae, z, zc, b, y, invd, omega, fixed,
               sc);
  return cudaGetLastError();
}
template cudaError_t launch_apply2_prolong<double>(const Dims&, const double*, const double*,
                                                   const double*, const double*, double*,
                                                   const double*, double, const uint8_t*, int,
                                                   const CgScalars*, cudaStream_t);
template cudaError_t launch_apply2_prolong<float>(const Dims&, const float*, const float*,
                                                  const float*, const float*, float*, const float*,
                                                  float, const uint8_t*, int, const CgScalars*,
                                                  cudaStream_t);

template <typename T>
cudaError_t launch_vcycle_tail(const TailArgs<T>& a, int nrhs, const CgScalars* sc,
                               cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kTailCluster, nrhs);
  cfg.blockDim = dim3(kTailThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kTailCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_vcycle_tail<T>, a, sc);
}
template cudaError_t launch_vcycle_tail<float>(const TailArgs<float>&, int, const CgScalars*,
                                               cudaStream_t);
template cudaError_t launch_vcycle_tail<double>(const TailArgs<double>&, int, const CgScalars*,
                                                cudaStream_t);

namespace {
int tail1_smem_limit() {
  static int lim = -1;
  if (lim < 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_vcycle_tail1<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin) != cudaSuccess ||
        cudaFuncSetAttribute(k_vcycle_tail1<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin) != cudaSuccess) {
      cudaGetLastError();
      optin = 0;
    }
    lim = optin;
  }
  return lim;
}
unsigned align16u(unsigned long long x) { return (unsigned)((x + 15ull) & ~15ull); }
}  // namespace


template <typename T>
bool tail1_layout(TailArgs<T>& a) {
  if (a.nc > kTail1MaxNc) return false;
  unsigned long long off = 0;
  for (int k = 0; k < a.nl; ++k) {
    const unsigned long long n = (unsigned long long)a.d[k].dofs();
    const unsigned long long m = (unsigned long long)a.d[k].elems();
    const bool coarsest = (k == a.nl - 1);
    a.off_m[k] = (unsigned)off;
    if (!coarsest) {
      if (!a.Aem[k]) return false;  // (no element-major copy of this level)
      off += align16u((unsigned long long)kAemStride * m * sizeof(T));
    }
    a.off_z[k] = (unsigned)off;
    off += align16u(n * sizeof(T));
    a.off_t[k] = (unsigned)off;
    if (!coarsest) off += align16u(n * sizeof(T));
    a.off_b[k] = (unsigned)off;
    off += align16u(n * sizeof(T));
    a.off_d[k] = (unsigned)off;
    if (!coarsest) off += align16u(n * sizeof(T));
    a.off_f[k] = (unsigned)off;
    off += align16u(n);
  }
  a.off_bar = (unsigned)off;
  off += 16;
  a.smem = (unsigned)off;
  return off > 0 && off <= (unsigned long long)tail1_smem_limit();
}
template bool tail1_layout<float>(TailArgs<float>&);
template bool tail1_layout<double>(TailArgs<double>&);

// Element-major copy of entry-major element matrices: Aem[e * kAemStride + r] = Ae[r * m + e]
// (r < 64; the 4 padding entries are not written and never read).
template <typename T>
__global__ void k_pack_element_major(long long m, const T* __restrict__ Ae, T* __restrict__ Aem) {
  pdl_prologue();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m * 64) return;
  const long long r = i / m, e = i - r * m;
  Aem[e * kAemStride + r] = Ae[i];
}

template <typename T>
cudaError_t launch_pack_element_major(long long m, const T* Ae, T* Aem, cudaStream_t st) {
  topo::launch(k_pack_element_major<T>, blocks_for(m * 64), kThreads, 0, st, m, Ae, Aem);
  return cudaGetLastError();
}
template cudaError_t launch_pack_element_major<float>(long long, const float*, float*, cudaStream_t);
template cudaError_t launch_pack_element_major<double>(long long, const double*, double*,
                                                       cudaStream_t);

template <typename T>
cudaError_t launch_vcycle_tail1(const TailArgs<T>& a, int nrhs, const CgScalars* sc,
                                cudaStream_t st) {
  topo::launch(k_vcycle_tail1<T>, dim3(nrhs), tail1_threads<T>(), a.smem, st, a, sc);
  return cudaGetLastError();
}
template cudaError_t launch_vcycle_tail1<float>(const TailArgs<float>&, int, const CgScalars*,
                                                cudaStream_t);
template cudaError_t launch_vcycle_tail1<double>(const TailArgs<double>&, int, const CgScalars*,
                                                 cudaStream_t);

// Whether a cluster of kTailCluster blocks of the fused kernel fits on this device (and the
// shared-memory limit of the single-block form, set here, outside any stream capture).
cudaError_t prepare_tail_kernels() {
  tail1_smem_limit();
  if (kTailCluster > 8) {
    cudaError_t e = cudaFuncSetAttribute(k_vcycle_tail<float>,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_vcycle_tail<double>,
                               cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  for (int p = 0; p < 2; ++p) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kTailCluster);
    cfg.blockDim = dim3(kTailThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kTailCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    cudaError_t e = p == 0 ? cudaOccupancyMaxActiveClusters(&clusters, k_vcycle_tail<float>, &cfg)
                           : cudaOccupancyMaxActiveClusters(&clusters, k_vcycle_tail<double>, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorNotSupported;
  }
  return cudaSuccess;
}

cudaError_t launch_inv_diag(const Dims& d, const double* K0, const double* x, const double* Ae,
                            const uint8_t* fixed, double* invd, cudaStream_t st) {
  if (d.dim == 2)
    topo::launch(k_inv_diag<2>, blocks_for(d.nodes()), kThreads, 0, st, d, K0, x, Ae, fixed, invd);
  else
    topo::launch(k_inv_diag<3>, blocks_for(d.nodes()), kThreads, 0, st, d, K0, x, Ae, fixed, invd);
  return cudaGetLastError();
}

cudaError_t launch_inv_diag32(const Dims& d, const float* Ae, const uint8_t* fixed, float* invd,
                              cudaStream_t st) {
  if (d.dim == 2)
    topo::launch(k_inv_diag32<2>, blocks_for(d.nodes()), kThreads, 0, st, d, Ae, fixed, invd);
  else
    topo::launch(k_inv_diag32<3>, blocks_for(d.nodes()), kThreads, 0, st, d, Ae, fixed, invd);
  return cudaGetLastError();
}

cudaError_t launch_element_energy(const Dims& d, const double* K0, const double* u,
                                  const double* lam, double* out, double scale, cudaStream_t st) {
  if (d.dim == 2)
    topo::launch(k_element_energy<2>, blocks_for(d.elems()), kThreads, 0, st, d, K0, u, lam, out, scale);
  else
    topo::launch(k_element_energy<3>, blocks_for(d.elems()), kThreads, 0, st, d, K0, u, lam, out, scale);
  return cudaGetLastError();
}

cudaError_t launch_convert_d2f(const double* a, float* b, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  topo::launch(k_d2f, blocks_for(n), kThreads, 0, st, a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_check_positive(const double* x, long long m, int* flag, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e != cudaSuccess || m <= 0) return e;
  topo::launch(k_check_positive, blocks_for(m), kThreads, 0, st, x, m, flag);
  return cudaGetLastError();
}

cudaError_t launch_convert_f2d(const float* a, double* b, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  topo::launch(k_f2d, blocks_for(n), kThreads, 0, st, a, b, n);
  return cudaGetLastError();
}

}  // namespace topo
