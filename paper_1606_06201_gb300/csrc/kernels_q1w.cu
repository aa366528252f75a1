// FP32 finest-level sweeps of the 2D Q1 grid with two node columns per lane: the operator
// K(x) v = sum_e x_e L_e^T K0 L_e v (Eq. (to), Sec. 7) inside the damped-Jacobi smoother,
// residual, restriction and prolongation of Algorithm MG (Sec. 5.1), with the element product of
// q1_common.cuh.
//
// Data movement.  A warp owns 62 consecutive output node columns and a strip of node rows.  Lane
// l holds the node columns a = 62 wc - 2 + 2 l and a + 1 and the element columns a and a + 1; it
// walks the strip row by row.  The right neighbour's node a + 2 of the new row comes by one
// shuffle pair, the left neighbour's contributions to node a (its second element's right-hand
// results) by two shuffle pairs, the left density by one shuffle: about 3.5 shuffles per output
// node against about 10 with one column per lane (kernels_q1.cu).  Each lane stages the rows it
// reads into a ring of four row slots in shared memory with asynchronous copies (cp.async, zero
// fill outside the grid), three rows ahead of their use: the rows in flight hold no registers, so
// the memory parallelism does not cost occupancy, and the boundary needs no branches.  The fixed-
// DOF mask is read from a copy with an even row stride (node pairs 4-byte aligned).  Each output
// node is summed from its four elements in the fixed order of the one-column kernels, and every
// per-node value is formed by the same expressions, so the outputs are the same bits; only the
// fused dot products (DOT 2) sum their terms in another order.  Lane 0 outputs node a + 1 only
// and lane 31 node a only (their other columns are halo).
#include "q1_common.cuh"
#include "topo_internal.cuh"

namespace topo {

namespace {

using namespace q1;

constexpr int kWCols = 62;   // output node columns per warp
constexpr int kWWarps = 4;   // warps per block
constexpr int kWMaxRows = 32;
constexpr int kRWCols = 30;  // coarse columns per warp of the residual-restriction kernel
constexpr int kWSlots = 4;   // row slots per warp (rows ey .. ey + 3)

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// Asynchronous global -> shared copy of `bytes` (4, 8 or 16); ok = false fills zeros and reads
// nothing (the source address is then only a placeholder inside the array).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_addr(dst)), "l"(src),
               "n"(BYTES), "r"(ok ? BYTES : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// MODE: 0 y = K v; 1 y = b - K v; 2 y = v + omega D^{-1} (b - K v); 3 y = omega D^{-1} b;
// 4 the first two sweeps from zero (z = omega D^{-1} b formed on the fly, then one sweep);
// 5 the prolongation t + P zc formed on the fly, then one sweep.  DOT 2: also r^T y against the
// FP64 residual.  The slot of one row holds, per lane: v (or t) of its two nodes, b, the coarse
// values of MODE 5, the FP64 residual (DOT 2), the densities of elements a, a + 1 (and a - 1 on
// lane 0), and the mask bytes of the node pair.
template <typename T, int MODE, int DOT>
struct WLayout {
  using V2 = typename Vec2<T>::type;
  static constexpr bool kV = MODE <= 2 || MODE == 5;
  static constexpr bool kB = MODE != 0;
  static constexpr bool kZ = MODE == 5;
  static constexpr bool kR = DOT == 2;
  static constexpr int kOffV = 0;
  static constexpr int kOffB = kOffV + (kV ? 2 * 32 * (int)sizeof(V2) : 0);
  static constexpr int kOffZ = kOffB + (kB ? 2 * 32 * (int)sizeof(V2) : 0);
  static constexpr int kOffR = kOffZ + (kZ ? 4 * 32 * (int)sizeof(V2) : 0);
  static constexpr int kOffX = kOffR + (kR ? 2 * 32 * (int)sizeof(double2) : 0);
  static constexpr int kOffF = kOffX + 3 * 32 * (int)sizeof(T);
  static constexpr int kSlot = (kOffF + 32 * 4 + 15) / 16 * 16;
  static constexpr int kWarp = kSlot * kWSlots;
};

// One row of a lane, read back from its slot.
template <typename T>
struct WRow {
  using V2 = typename Vec2<T>::type;
  V2 v0, v1, b0, b1, z0, z1, w0, w1;
  double2 r0, r1;
  T xA, xB, xL;
  unsigned f;  // mask bytes: x, y of node a, then x, y of node a + 1
};

template <typename T, int MODE, int DOT>
struct WCtx {
  using V2 = typename Vec2<T>::type;
  using L = WLayout<T, MODE, DOT>;
  int nx, ny, a, rs, crs, lane;
  bool n0, n1, e0, e1, xl0;
  const T* x;
  const V2* v2;
  const V2* b2;
  const V2* zc2;
  const double2* rd2;
  const unsigned* fpad;  // mask node pairs, row stride (nx + 2) / 2
  char* ring;            // this warp's slots

  __device__ __forceinline__ char* slot(int r) const { return ring + ((r + kWSlots) & (kWSlots - 1)) * L::kSlot; }

  // Stage node row r (and element row r) into its slot; one commit group per row.  want = false
  // (a row the strip does not read) fills the slot with zeros and reads nothing.
  __device__ __forceinline__ void issue(int r, bool want = true) const {
    char* sl = slot(r);
    const bool row = want && r >= 0 && r <= ny, el = row && r < ny;
    const int rr = row ? r : 0, re = el ? r : 0;
    const int nd = a + rs * rr;
    const long long NN = (long long)rs * (ny + 1), NC = (long long)crs * (ny / 2 + 1);
    const bool k0 = row && n0 && TOPO_IN(nd, NN), k1 = row && n1 && TOPO_IN(nd + 1, NN);
    if (L::kV) {
      cp_async<sizeof(V2)>(sl + L::kOffV + lane * sizeof(V2), v2 + (k0 ? nd : 0), k0);
      cp_async<sizeof(V2)>(sl + L::kOffV + (32 + lane) * sizeof(V2), v2 + (k1 ? nd + 1 : 0), k1);
    }
    if (L::kB) {
      cp_async<sizeof(V2)>(sl + L::kOffB + lane * sizeof(V2), b2 + (k0 ? nd : 0), k0);
      cp_async<sizeof(V2)>(sl + L::kOffB + (32 + lane) * sizeof(V2), b2 + (k1 ? nd + 1 : 0), k1);
    }
    if (L::kZ) {
      const int i0 = k0 ? a >> 1 : 0, q0 = rr >> 1, q1 = (rr + 1) >> 1;
      const bool odd = (r & 1) != 0;
      const bool z0 = k0 && TOPO_IN(i0 + crs * q0, NC), z1 = k1 && TOPO_IN(i0 + 1 + crs * q0, NC);
      const bool z2 = k0 && odd && TOPO_IN(i0 + crs * q1, NC);
      const bool z3 = k1 && odd && TOPO_IN(i0 + 1 + crs * q1, NC);
      cp_async<sizeof(V2)>(sl + L::kOffZ + lane * sizeof(V2), zc2 + (z0 ? i0 + crs * q0 : 0), z0);
      cp_async<sizeof(V2)>(sl + L::kOffZ + (32 + lane) * sizeof(V2),
                           zc2 + (z1 ? i0 + 1 + crs * q0 : 0), z1);
      cp_async<sizeof(V2)>(sl + L::kOffZ + (64 + lane) * sizeof(V2),
                           zc2 + (z2 ? i0 + crs * q1 : 0), z2);
      cp_async<sizeof(V2)>(sl + L::kOffZ + (96 + lane) * sizeof(V2),
                           zc2 + (z3 ? i0 + 1 + crs * q1 : 0), z3);
    }
    if (L::kR) {
      cp_async<16>(sl + L::kOffR + lane * 16, rd2 + (k0 ? nd : 0), k0);
      cp_async<16>(sl + L::kOffR + (32 + lane) * 16, rd2 + (k1 ? nd + 1 : 0), k1);
    }
    const long long M = (long long)nx * ny, NF = (long long)((nx + 2) >> 1) * (ny + 1);
    const bool xa = el && e0 && TOPO_IN(a + nx * re, M), xb = el && e1 && TOPO_IN(a + 1 + nx * re, M);
    const bool xc = el && xl0 && (MODE != 4 || lane != 0 || TOPO_IN(a - 1 + nx * re, M));
    cp_async<sizeof(T)>(sl + L::kOffX + lane * sizeof(T), x + (xa ? a + nx * re : 0), xa);
    cp_async<sizeof(T)>(sl + L::kOffX + (32 + lane) * sizeof(T), x + (xb ? a + 1 + nx * re : 0), xb);
    if (MODE == 4 && lane == 0)
      cp_async<sizeof(T)>(sl + L::kOffX + 64 * sizeof(T), x + (xc ? a - 1 + nx * re : 0), xc);
    const bool kf = k0 && TOPO_IN((a >> 1) + ((nx + 2) >> 1) * rr, NF);
    cp_async<4>(sl + L::kOffF + lane * 4, fpad + (kf ? (a >> 1) + ((nx + 2) >> 1) * rr : 0), kf);
    cp_commit();
  }

  __device__ __forceinline__ WRow<T> read(int r) const {
    const char* sl = slot(r);
    WRow<T> R;
    V2 zero;
    zero.x = T(0);
    zero.y = T(0);
    R.v0 = R.v1 = R.b0 = R.b1 = R.z0 = R.z1 = R.w0 = R.w1 = zero;
    R.r0 = R.r1 = make_double2(0.0, 0.0);
    if (L::kV) {
      R.v0 = *reinterpret_cast<const V2*>(sl + L::kOffV + lane * sizeof(V2));
      R.v1 = *reinterpret_cast<const V2*>(sl + L::kOffV + (32 + lane) * sizeof(V2));
    }
    if (L::kB) {
      R.b0 = *reinterpret_cast<const V2*>(sl + L::kOffB + lane * sizeof(V2));
      R.b1 = *reinterpret_cast<const V2*>(sl + L::kOffB + (32 + lane) * sizeof(V2));
    }
    if (L::kZ) {
      R.z0 = *reinterpret_cast<const V2*>(sl + L::kOffZ + lane * sizeof(V2));
      R.z1 = *reinterpret_cast<const V2*>(sl + L::kOffZ + (32 + lane) * sizeof(V2));
      R.w0 = *reinterpret_cast<const V2*>(sl + L::kOffZ + (64 + lane) * sizeof(V2));
      R.w1 = *reinterpret_cast<const V2*>(sl + L::kOffZ + (96 + lane) * sizeof(V2));
    }
    if (L::kR) {
      R.r0 = *reinterpret_cast<const double2*>(sl + L::kOffR + lane * 16);
      R.r1 = *reinterpret_cast<const double2*>(sl + L::kOffR + (32 + lane) * 16);
    }
    R.xA = *reinterpret_cast<const T*>(sl + L::kOffX + lane * sizeof(T));
    R.xB = *reinterpret_cast<const T*>(sl + L::kOffX + (32 + lane) * sizeof(T));
    // (lane 0's own copy: a lane reads only what its own copies wrote)
    R.xL = (MODE == 4 && lane == 0) ? *reinterpret_cast<const T*>(sl + L::kOffX + 64 * sizeof(T)) : T(0);
    R.f = *reinterpret_cast<const unsigned*>(sl + L::kOffF + lane * 4);
    return R;
  }
};

// Input value of the sweep at node row r for the lane's two nodes (MODE 0-2: v; 3: none;
// 4: omega D^{-1} b, masked; 5: t + P zc, fixed DOFs keep t).  The expressions and their order are
// those of k_q1_fused and k_prolong_add.
template <typename T, int MODE>
__device__ __forceinline__ void w_input(const WRow<T>& R, int r, T omega, const Q1K<T>& k,
                                        T xsA, T xsB, T& dA, T& dB, typename Vec2<T>::type& o0,
                                        typename Vec2<T>::type& o1) {
  const unsigned f = R.f;
  if (MODE <= 2) {
    o0 = R.v0;
    o1 = R.v1;
  } else if (MODE == 3) {
    o0.x = o0.y = o1.x = o1.y = T(0);
  } else if (MODE == 4) {
    dA = xsA > T(0) ? recip_rn(k.kd * xsA) : T(1);
    dB = xsB > T(0) ? recip_rn(k.kd * xsB) : T(1);
    const T wA = mul_rn(omega, dA), wB = mul_rn(omega, dB);
    o0.x = (f & 0xffu) ? T(0) : mul_rn(wA, R.b0.x);
    o0.y = (f & 0xff00u) ? T(0) : mul_rn(wA, R.b0.y);
    o1.x = (f & 0xff0000u) ? T(0) : mul_rn(wB, R.b1.x);
    o1.y = (f & 0xff000000u) ? T(0) : mul_rn(wB, R.b1.y);
  } else {
    // node a (even column): weights 1 (even row) or 1/2 (odd row), coarse column a/2 only;
    // node a + 1 (odd column): weights 1/2 or 1/4, coarse columns a/2 and a/2 + 1
    const T wy = (r & 1) ? T(0.5) : T(1);
    const T w0 = T(1) * wy * T(1), w1 = T(0.5) * wy * T(1);
    T ax = fma(w0, R.z0.x, T(0)), ay = fma(w0, R.z0.y, T(0));
    T bx = fma(w1, R.z0.x, T(0)), by = fma(w1, R.z0.y, T(0));
    bx = fma(w1, R.z1.x, bx);
    by = fma(w1, R.z1.y, by);
    if (r & 1) {
      ax = fma(w0, R.w0.x, ax);
      ay = fma(w0, R.w0.y, ay);
      bx = fma(w1, R.w0.x, bx);
      by = fma(w1, R.w0.y, by);
      bx = fma(w1, R.w1.x, bx);
      by = fma(w1, R.w1.y, by);
    }
    o0 = R.v0;
    o1 = R.v1;
    if (!(f & 0xffu)) o0.x = R.v0.x + ax;
    if (!(f & 0xff00u)) o0.y = R.v0.y + ay;
    if (!(f & 0xff0000u)) o1.x = R.v1.x + bx;
    if (!(f & 0xff000000u)) o1.y = R.v1.y + by;
  }
}

template <typename T>
__device__ __forceinline__ T dinv_of(const Q1K<T>& k, T xs) {
  return xs > T(0) ? recip_rn(k.kd * xs) : T(1);
}

template <typename T, int MODE>
__device__ __forceinline__ T w_out(T q, T bin, T vin, T omega, T dinv) {
  if (MODE == 0) return q;
  if (MODE == 1) return bin - q;
  if (MODE == 3) return omega * dinv * bin;
  return fma(omega * dinv, bin - q, vin);
}

template <typename T, int MODE, int DOT>
__global__ void __launch_bounds__(kWWarps * 32) k_q1w(int nx, int ny, int rows, Q1K<T> k,
                                                      const T* __restrict__ x,
                                                      const T* __restrict__ v,
                                                      const T* __restrict__ zc,
                                                      const T* __restrict__ b,
                                                      T* __restrict__ y, T omega,
                                                      const unsigned* __restrict__ fpad,
                                                      CgScalars* sc, double* partials,
                                                      unsigned* counters,
                                                      const double* __restrict__ rdot) {
  pdl_prologue();
  using V2 = typename Vec2<T>::type;
  using L = WLayout<T, MODE, DOT>;
  extern __shared__ __align__(16) char w_smem[];
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const long long n = 2LL * (nx + 1) * (ny + 1);
  if (MODE <= 2 || MODE == 5) v += rhs * n;
  if (MODE != 0) b += rhs * n;
  y += rhs * n;
  if (MODE == 5) zc += rhs * 2LL * (nx / 2 + 1) * (ny / 2 + 1);
  if (DOT == 2) rdot += rhs * n;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kWWarps + (threadIdx.x >> 5);
  const int ncolw = (nx + 2 + kWCols - 1) / kWCols;
  const int nstrip = (ny + 1 + rows - 1) / rows;
  const int wc = gw % ncolw, ws = gw / ncolw;
  double part = 0.0;
  if (ws < nstrip) {
    WCtx<T, MODE, DOT> C;
    C.nx = nx;
    C.ny = ny;
    C.lane = lane;
    C.a = kWCols * wc - 2 + 2 * lane;
    C.rs = nx + 1;
    C.crs = nx / 2 + 1;
    const int a = C.a;
    C.n0 = (a >= 0 && a <= nx);
    C.n1 = (a + 1 >= 0 && a + 1 <= nx);
    C.e0 = (a >= 0 && a < nx);
    C.e1 = (a + 1 >= 0 && a + 1 < nx);
    C.xl0 = (lane == 0 && a - 1 >= 0 && a - 1 < nx);
    C.x = x;
    C.v2 = reinterpret_cast<const V2*>(v);
    C.b2 = reinterpret_cast<const V2*>(b);
    C.zc2 = reinterpret_cast<const V2*>(zc);
    C.rd2 = reinterpret_cast<const double2*>(rdot);
    C.fpad = fpad;
    C.ring = w_smem + (threadIdx.x >> 5) * L::kWarp;
    const bool out0 = lane >= 1 && C.n0, out1 = lane <= 30 && C.n1;
    const int j0 = ws * rows;
    const int j1 = min(j0 + rows, ny + 1);
    V2 zero;
    zero.x = T(0);
    zero.y = T(0);
    C.issue(j0 - 1);
    C.issue(j0);
    C.issue(j0 + 1);
    // MODE 4 forms the input of node row j0 - 1 from the densities of element rows j0 - 2, j0 - 1
    T pmA = T(0), pmB = T(0);
    if (MODE == 4 && j0 - 2 >= 0) {
      const int r = j0 - 2;
      const T xa = C.e0 ? x[a + nx * r] : T(0), xb = C.e1 ? x[a + 1 + nx * r] : T(0);
      const T xlo = C.xl0 ? x[a - 1 + nx * r] : T(0);
      const T xl = shfl_up1(xb);
      pmA = xa + (lane >= 1 ? xl : xlo);
      pmB = xb + xa;
    }
    cp_wait<2>();  // row j0 - 1 is in
    WRow<T> R0 = C.read(j0 - 1);
    T pcA = T(0), pcB = T(0);
    if (MODE == 4) {
      const T xl = shfl_up1(R0.xB);
      pcA = R0.xA + (lane >= 1 ? xl : R0.xL);
      pcB = R0.xB + R0.xA;
    }
    T dinA = T(0), dinB = T(0);  // MODE 4: the diagonal of the last input row
    V2 pb0 = zero, pb1 = zero;
    if (j0 - 1 >= 0) w_input<T, MODE>(R0, j0 - 1, omega, k, pmA + pcA, pmB + pcB, dinA, dinB, pb0, pb1);
    if (!C.n0) pb0 = zero;
    if (!C.n1) pb1 = zero;
    V2 pbR;
    pbR.x = shfl_dn(pb0.x);
    pbR.y = shfl_dn(pb0.y);
    T cuA = T(0), cvA = T(0), cuB = T(0), cvB = T(0);
    T xcA = T(0), xcB = T(0);  // MODE 2, 3, 5: the density pairs of the element row below
    for (int ey = j0 - 1; ey < j1; ++ey) {
      C.issue(ey + 3, ey + 3 <= ny && ey + 2 < j1);
      cp_wait<2>();  // rows ey and ey + 1 are in
      const WRow<T> R = C.read(ey);      // node row ey (b, mask), element row ey (densities)
      const WRow<T> N = C.read(ey + 1);  // node row ey + 1
      const T dA_row = dinA, dB_row = dinB;
      T pnA = T(0), pnB = T(0);
      if (MODE == 4) {
        const T xl = shfl_up1(N.xB);
        pnA = N.xA + (lane >= 1 ? xl : N.xL);
        pnB = N.xB + N.xA;
      }
      V2 pt0 = zero, pt1 = zero;
      if (ey + 1 <= ny) w_input<T, MODE>(N, ey + 1, omega, k, pcA + pnA, pcB + pnB, dinA, dinB, pt0, pt1);
      if (!C.n0) pt0 = zero;
      if (!C.n1) pt1 = zero;
      V2 ptR;
      ptR.x = shfl_dn(pt0.x);
      ptR.y = shfl_dn(pt0.y);
      const T xeA = R.xA, xeB = R.xB;  // zero outside the grid (zero fill)
      T ruA[4], rvA[4], ruB[4], rvB[4];
      if (MODE != 3) {
        {
          const T uu[4] = {pb0.x, pb1.x, pt1.x, pt0.x};
          const T vv[4] = {pb0.y, pb1.y, pt1.y, pt0.y};
          q1_element<T>(k, xeA, uu, vv, ruA, rvA);
        }
        {
          const T uu[4] = {pb1.x, pbR.x, ptR.x, pt1.x};
          const T vv[4] = {pb1.y, pbR.y, ptR.y, pt1.y};
          q1_element<T>(k, xeB, uu, vv, ruB, rvB);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) ruA[q] = rvA[q] = ruB[q] = rvB[q] = T(0);
      }
      const T l1u = shfl_up1(ruB[1]), l1v = shfl_up1(rvB[1]);
      const T l2u = shfl_up1(ruB[2]), l2v = shfl_up1(rvB[2]);
      T xpA = T(0), xpB = T(0);
      if (MODE == 2 || MODE == 3 || MODE == 5) {
        const T xl = shfl_up1(xeB);
        xpA = xeA + (lane >= 1 ? xl : T(0));
        xpB = xeB + xeA;
      }
      if (ey >= j0) {
        T dA = T(0), dB = T(0);
        if (MODE == 2 || MODE == 3 || MODE == 5) {
          dA = dinv_of(k, xcA + xpA);
          dB = dinv_of(k, xcB + xpB);
        } else if (MODE == 4) {
          dA = dA_row;
          dB = dB_row;
        }
        const int node = a + C.rs * ey;
        const unsigned f = R.f;
        if (out0) {
          const T qu = cuA + ruA[0] + l1u, qv = cvA + rvA[0] + l1v;
          V2 o;
          o.x = w_out<T, MODE>(qu, R.b0.x, pb0.x, omega, dA);
          o.y = w_out<T, MODE>(qv, R.b0.y, pb0.y, omega, dA);
          if (f & 0xffu) o.x = T(0);
          if (f & 0xff00u) o.y = T(0);
          if (TOPO_IN(node, (long long)C.rs * (C.ny + 1))) reinterpret_cast<V2*>(y)[node] = o;
          if (DOT == 1) part = fma(double_of(pb0.x), double_of(o.x), fma(double_of(pb0.y), double_of(o.y), part));
          if (DOT == 2) part = fma(R.r0.x, double_of(o.x), fma(R.r0.y, double_of(o.y), part));
        }
        if (out1) {
          const T qu = cuB + ruB[0] + ruA[1], qv = cvB + rvB[0] + rvA[1];
          V2 o;
          o.x = w_out<T, MODE>(qu, R.b1.x, pb1.x, omega, dB);
          o.y = w_out<T, MODE>(qv, R.b1.y, pb1.y, omega, dB);
          if (f & 0xff0000u) o.x = T(0);
          if (f & 0xff000000u) o.y = T(0);
          if (TOPO_IN(node + 1, (long long)C.rs * (C.ny + 1))) reinterpret_cast<V2*>(y)[node + 1] = o;
          if (DOT == 1) part = fma(double_of(pb1.x), double_of(o.x), fma(double_of(pb1.y), double_of(o.y), part));
          if (DOT == 2) part = fma(R.r1.x, double_of(o.x), fma(R.r1.y, double_of(o.y), part));
        }
      }
      xcA = xpA;
      xcB = xpB;
      cuA = ruA[3] + l2u;
      cvA = rvA[3] + l2v;
      cuB = ruB[3] + ruA[2];
      cvB = rvB[3] + rvA[2];
      pcA = pnA;
      pcB = pnB;
      pb0 = pt0;
      pb1 = pt1;
      pbR = ptR;
    }
    cp_wait<0>();  // no copy outlives the warp's slots
  }
  if (DOT) q1_finish_dot<DOT>(part, rhs, sc, partials, counters);
}

// b_c = P^T (b - K(x) v) in one pass (the residual of k_q1w<T, 1, 0>, never stored), combined by
// the 9-point full weighting in the order of k_restrict: per coarse node the fine rows 2J - 1, 2J,
// 2J + 1 and in each row the columns 2I - 1, 2I, 2I + 1.  Lane l (1..30) of warp wc owns the
// coarse column I = 30 wc + l - 1 (fine node a = 2I, with a + 1 its own and a - 1 from lane
// l - 1); the warp walks the fine rows 2 J0 - 1 .. 2 J1 - 1 of its strip of coarse rows.
template <typename T>
__global__ void __launch_bounds__(kWWarps * 32) k_q1w_resrestrict(int nx, int ny, int crows,
                                                                  Q1K<T> k,
                                                                  const T* __restrict__ x,
                                                                  const T* __restrict__ v,
                                                                  const T* __restrict__ b,
                                                                  T* __restrict__ bc,
                                                                  const unsigned* __restrict__ fpad,
                                                                  const uint8_t* __restrict__ fixed_c,
                                                                  const CgScalars* sc) {
  pdl_prologue();
  using V2 = typename Vec2<T>::type;
  using L = WLayout<T, 1, 0>;
  extern __shared__ __align__(16) char w_smem[];
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const long long n = 2LL * (nx + 1) * (ny + 1);
  const int cnx = nx / 2, cny = ny / 2;
  v += rhs * n;
  b += rhs * n;
  bc += rhs * 2LL * (cnx + 1) * (cny + 1);
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kWWarps + (threadIdx.x >> 5);
  const int ncolw = (cnx + 1 + kRWCols - 1) / kRWCols;
  const int nstrip = (cny + 1 + crows - 1) / crows;
  const int wc = gw % ncolw, ws = gw / ncolw;
  if (ws >= nstrip) return;
  WCtx<T, 1, 0> C;
  C.nx = nx;
  C.ny = ny;
  C.lane = lane;
  C.a = 2 * kRWCols * wc - 2 + 2 * lane;
  C.rs = nx + 1;
  C.crs = cnx + 1;
  const int a = C.a;
  C.n0 = (a >= 0 && a <= nx);
  C.n1 = (a + 1 >= 0 && a + 1 <= nx);
  C.e0 = (a >= 0 && a < nx);
  C.e1 = (a + 1 >= 0 && a + 1 < nx);
  C.xl0 = false;
  C.x = x;
  C.v2 = reinterpret_cast<const V2*>(v);
  C.b2 = reinterpret_cast<const V2*>(b);
  C.zc2 = nullptr;
  C.rd2 = nullptr;
  C.fpad = fpad;
  C.ring = w_smem + (threadIdx.x >> 5) * L::kWarp;
  const bool out0 = lane >= 1 && C.n0, out1 = lane <= 30 && C.n1;
  const bool own = lane >= 1 && lane <= 30 && C.n0;
  const int I = a >> 1;
  const int J0 = ws * crows, J1 = min(J0 + crows, cny + 1);
  const int j0 = max(2 * J0 - 1, 0), j1 = min(2 * J1 - 1, ny) + 1;  // fine rows [j0, j1)
  V2 zero;
  zero.x = T(0);
  zero.y = T(0);
  C.issue(j0 - 1);
  C.issue(j0);
  C.issue(j0 + 1);
  cp_wait<2>();
  const WRow<T> R0 = C.read(j0 - 1);
  V2 pb0 = R0.v0, pb1 = R0.v1;  // zero outside the grid
  V2 pbR;
  pbR.x = shfl_dn(pb0.x);
  pbR.y = shfl_dn(pb0.y);
  T cuA = T(0), cvA = T(0), cuB = T(0), cvB = T(0);
  T ax = T(0), ay = T(0);  // the full-weighting sums of the coarse row in progress
  for (int ey = j0 - 1; ey < j1; ++ey) {
    C.issue(ey + 3, ey + 3 <= ny && ey + 2 < j1);
    cp_wait<2>();
    const WRow<T> R = C.read(ey);
    const WRow<T> N = C.read(ey + 1);
    const V2 pt0 = N.v0, pt1 = N.v1;  // zero beyond the grid
    V2 ptR;
    ptR.x = shfl_dn(pt0.x);
    ptR.y = shfl_dn(pt0.y);
    T ruA[4], rvA[4], ruB[4], rvB[4];
    {
      const T uA[4] = {pb0.x, pb1.x, pt1.x, pt0.x}, vA[4] = {pb0.y, pb1.y, pt1.y, pt0.y};
      q1_element<T>(k, R.xA, uA, vA, ruA, rvA);
      const T uB[4] = {pb1.x, pbR.x, ptR.x, pt1.x}, vB[4] = {pb1.y, pbR.y, ptR.y, pt1.y};
      q1_element<T>(k, R.xB, uB, vB, ruB, rvB);
    }
    const T l1u = shfl_up1(ruB[1]), l1v = shfl_up1(rvB[1]);
    const T l2u = shfl_up1(ruB[2]), l2v = shfl_up1(rvB[2]);
    if (ey >= j0) {  // residual of node row ey (warp-uniform), then its share of P^T r
      V2 r0 = zero, r1 = zero;
      const unsigned f = R.f;
      if (out0) {
        r0.x = R.b0.x - (cuA + ruA[0] + l1u);
        r0.y = R.b0.y - (cvA + rvA[0] + l1v);
        if (f & 0xffu) r0.x = T(0);
        if (f & 0xff00u) r0.y = T(0);
      }
      if (out1) {
        r1.x = R.b1.x - (cuB + ruB[0] + ruA[1]);
        r1.y = R.b1.y - (cvB + rvB[0] + rvA[1]);
        if (f & 0xff0000u) r1.x = T(0);
        if (f & 0xff000000u) r1.y = T(0);
      }
      const T rlx = shfl_up1(r1.x), rly = shfl_up1(r1.y);  // node a - 1
      auto row_terms = [&](T wy, T& sx, T& sy) {
        if (a - 1 >= 0) {
          const T w = wy * T(0.5);
          sx = fma(w, rlx, sx);
          sy = fma(w, rly, sy);
        }
        sx = fma(wy, r0.x, sx);
        sy = fma(wy, r0.y, sy);
        if (a + 1 <= nx) {
          const T w = wy * T(0.5);
          sx = fma(w, r1.x, sx);
          sy = fma(w, r1.y, sy);
        }
      };
      auto write = [&](int J, T sx, T sy) {
        const long long cid = 2LL * (I + (long long)(cnx + 1) * J);
        V2 o;
        o.x = fixed_c[cid] ? T(0) : sx;
        o.y = fixed_c[cid + 1] ? T(0) : sy;
        reinterpret_cast<V2*>(bc)[cid >> 1] = o;
      };
      if (own) {
        if ((ey & 1) == 0) {  // fine row 2J: the middle row of coarse row J
          const int J = ey >> 1;
          row_terms(T(1), ax, ay);
          if (ey == ny && J >= J0 && J < J1) write(J, ax, ay);
        } else {  // fine row 2J + 1: the last row of coarse row J, the first of J + 1
          const int J = ey >> 1;
          if (J >= J0) {
            row_terms(T(1) * T(0.5), ax, ay);
            write(J, ax, ay);
          }
          ax = T(0);
          ay = T(0);
          row_terms(T(1) * T(0.5), ax, ay);
        }
      }
    }
    cuA = ruA[3] + l2u;
    cvA = rvA[3] + l2v;
    cuB = ruB[3] + ruA[2];
    cvB = rvB[3] + rvA[2];
    pb0 = pt0;
    pb1 = pt1;
    pbR = ptR;
  }
  cp_wait<0>();
}

#ifndef TOPO_Q1W_WARPS_PER_SM
#define TOPO_Q1W_WARPS_PER_SM 16
#endif

// Strip height: about one wave of warps (152 SMs x TOPO_Q1W_WARPS_PER_SM), long enough to
// amortise the recomputed first element row of each strip.
int w_rows(int nx, int ny, int want = 0) {
  if (want >= 2) return want < kWMaxRows ? want : kWMaxRows;
  const long long ncolw = (nx + 2 + kWCols - 1) / kWCols;
  const long long target = 152LL * TOPO_Q1W_WARPS_PER_SM;
  long long r = (ncolw * (ny + 1) + target - 1) / target;
  if (r < 2) r = 2;
  if (r > kWMaxRows) r = kWMaxRows;
  return (int)r;
}

unsigned w_blocks(int nx, int ny, int want = 0) {
  const int rows = w_rows(nx, ny, want);
  const long long warps = (long long)((nx + 2 + kWCols - 1) / kWCols) * ((ny + 1 + rows - 1) / rows);
  return (unsigned)((warps + kWWarps - 1) / kWWarps);
}

template <int MODE, int DOT>
void w_launch(int nx, int ny, const Q1Coef& coef, const float* x, const float* v, const float* zc,
              const float* b, float* y, float omega, const unsigned* fpad, int nrhs,
              CgScalars* sc, double* partials, unsigned* counters, const double* rdot,
              cudaStream_t st, int want) {
  dim3 grid(w_blocks(nx, ny, want), nrhs);
  const size_t smem = (size_t)kWWarps * WLayout<float, MODE, DOT>::kWarp;
  static_assert((size_t)kWWarps * WLayout<float, MODE, DOT>::kWarp <= 48 * 1024,
                "row slots of a block fit the default shared-memory limit");
  topo::launch(k_q1w<float, MODE, DOT>, grid, kWWarps * 32, smem, st, nx, ny,
               w_rows(nx, ny, want), coef_cast<float>(coef), x, v, zc, b, y, omega, fpad, sc,
               partials, counters, rdot);
}

}  // namespace

long long q1w_partial_blocks(int nx, int ny) { return w_blocks(nx, ny); }

cudaError_t launch_q1w_apply(int nx, int ny, int mode, const Q1Coef& coef, const float* x,
                             const float* v, const float* b, float* y, float omega,
                             const unsigned* fixed, int nrhs, const CgScalars* sc,
                             cudaStream_t st, int rows) {
  CgScalars* scm = const_cast<CgScalars*>(sc);
  switch (mode) {
    case 0:
      w_launch<0, 0>(nx, ny, coef, x, v, nullptr, b, y, omega, fixed, nrhs, scm, nullptr, nullptr,
                     nullptr, st, rows);
      break;
    case 1:
      w_launch<1, 0>(nx, ny, coef, x, v, nullptr, b, y, omega, fixed, nrhs, scm, nullptr, nullptr,
                     nullptr, st, rows);
      break;
    case 2:
      w_launch<2, 0>(nx, ny, coef, x, v, nullptr, b, y, omega, fixed, nrhs, scm, nullptr, nullptr,
                     nullptr, st, rows);
      break;
    default:
      w_launch<3, 0>(nx, ny, coef, x, v, nullptr, b, y, omega, fixed, nrhs, scm, nullptr, nullptr,
                     nullptr, st, rows);
  }
  return cudaGetLastError();
}

cudaError_t launch_q1w_fused(int nx, int ny, int mode, const Q1Coef& coef, const float* x,
                             const float* t, const float* zc, const float* b, float* y,
                             float omega, const unsigned* fixed, int nrhs, const CgScalars* sc,
                             cudaStream_t st, int rows) {
  CgScalars* scm = const_cast<CgScalars*>(sc);
  if (mode == 4)
    w_launch<4, 0>(nx, ny, coef, x, nullptr, nullptr, b, y, omega, fixed, nrhs, scm, nullptr,
                   nullptr, nullptr, st, rows);
  else
    w_launch<5, 0>(nx, ny, coef, x, t, zc, b, y, omega, fixed, nrhs, scm, nullptr, nullptr,
                   nullptr, st, rows);
  return cudaGetLastError();
}

cudaError_t launch_q1w_smooth_beta(int nx, int ny, const Q1Coef& coef, const float* x,
                                   const float* v, const float* b, float* y, float omega,
                                   const unsigned* fixed, int nrhs, const double* r,
                                   double* partials, unsigned* counters, CgScalars* sc,
                                   cudaStream_t st, int rows) {
  w_launch<2, 2>(nx, ny, coef, x, v, nullptr, b, y, omega, fixed, nrhs, sc, partials, counters, r,
                 st, rows);
  return cudaGetLastError();
}

cudaError_t launch_q1w_resrestrict(int nx, int ny, const Q1Coef& coef, const float* x,
                                   const float* v, const float* b, float* bc,
                                   const unsigned* fixed, const uint8_t* fixed_c, int nrhs,
                                   const CgScalars* sc, cudaStream_t st, int rows) {
  const int cnx = nx / 2, cny = ny / 2;
  const long long ncolw = (cnx + 1 + kRWCols - 1) / kRWCols;
  const long long target = 152LL * TOPO_Q1W_WARPS_PER_SM;
  long long crows = rows >= 2 ? rows / 2 : (ncolw * (cny + 1) + target - 1) / target;
  if (crows < 1) crows = 1;
  if (crows > kWMaxRows / 2) crows = kWMaxRows / 2;
  const long long warps = ncolw * ((cny + 1 + crows - 1) / crows);
  dim3 grid((unsigned)((warps + kWWarps - 1) / kWWarps), nrhs);
  const size_t smem = (size_t)kWWarps * WLayout<float, 1, 0>::kWarp;
  topo::launch(k_q1w_resrestrict<float>, grid, kWWarps * 32, smem, st, nx, ny, (int)crows,
               coef_cast<float>(coef), x, v, b, bc, fixed, fixed_c, sc);
  return cudaGetLastError();
}

}  // namespace topo
