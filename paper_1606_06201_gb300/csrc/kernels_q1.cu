// Finest-level operator of the 2D Q1 grid, K(x) v = sum_e x_e L_e^T K0 L_e v (Eq. (to), Sec. 7),
// specialised for square plane-stress elements.
//
// The element product (two butterflies in the (1, xi, eta, xi eta) basis) is in q1_common.cuh.
//
// Data movement.  A warp owns 30 consecutive node columns and a strip of node rows.  Lane l holds
// node column c = i0 - 1 + l and element column c; it walks the strip row by row, loading one node
// of v and one density per row (coalesced), gets its right neighbour's nodes with a shuffle, forms
// its element's eight results, passes the right-hand results to the next lane with a shuffle and
// carries the top results in registers to the next row.  Each output node is summed from its four
// elements in a fixed order (deterministic, no atomics); lanes 0 and 31 only supply halo values.
// The Jacobi diagonal K0_ii sum_{e at node} x_e is formed on the fly from the same densities.
#include "pairs.cuh"
#include "q1_common.cuh"
#include "topo_internal.cuh"

namespace topo {

namespace {

constexpr int kQ1Cols = 30;   // output node columns per warp
constexpr int kQ1MaxRows = 16;  // output node rows per warp strip (at most)
constexpr int kQ1Warps = 8;   // warps per block

using namespace q1;

// MODE 0: y = K v; 1: y = b - K v; 2: y = v + omega D^{-1} (b - K v); 3: y = omega D^{-1} b.
// DOT 1 (MODE 0, FP64): also p^T q with the last-block finalisation alpha = r^T y / p^T q.
// DOT 2 (MODE 2, the last smoothing sweep of the preconditioner): also r~^T y~ against the FP64 CG
// residual rdot, with the last-block finalisation beta = r~^T y~ / r^T y of Algorithm PCG.
template <typename T, int MODE, int DOT>
__global__ void __launch_bounds__(kQ1Warps * 32) k_q1_sweep(int nx, int ny, int rows, Q1K<T> k,
                                                             const T* __restrict__ x,
                                                             const T* __restrict__ v,
                                                             const T* __restrict__ b,
                                                             T* __restrict__ y, T omega,
                                                             const uint8_t* __restrict__ fixed,
                                                             CgScalars* sc, double* partials,
                                                             unsigned* counters,
                                                             const double* __restrict__ rdot) {
  pdl_prologue();
  using V2 = typename Vec2<T>::type;
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const long long n = 2LL * (nx + 1) * (ny + 1);
  v += rhs * n;
  y += rhs * n;
  if (DOT == 2) rdot += rhs * n;
  if (MODE == 1 || MODE == 2 || MODE == 3) b += rhs * n;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kQ1Warps + (threadIdx.x >> 5);
  const int ncolw = (nx + 1 + kQ1Cols - 1) / kQ1Cols;
  const int nstrip = (ny + 1 + rows - 1) / rows;
  const int wc = gw % ncolw, ws = gw / ncolw;
  double part = 0.0;
  if (ws < nstrip) {
    const int c = wc * kQ1Cols - 1 + lane;           // node column and element column of the lane
    const bool col_ok = (c >= 0 && c <= nx);
    const bool out_lane = (lane >= 1 && lane <= kQ1Cols && col_ok);
    const bool el_col = (lane <= kQ1Cols && c >= 0 && c < nx);
    const int j0 = ws * rows;
    const int j1 = min(j0 + rows, ny + 1);
    const V2* v2 = reinterpret_cast<const V2*>(v);
    const V2* b2 = reinterpret_cast<const V2*>(b);
    const int rs = nx + 1;  // node row stride (grids hold < 2^31 DOFs: 32-bit indices)
    V2 zero;
    zero.x = T(0);
    zero.y = T(0);
    V2 pb = zero;
    const long long NN = (long long)rs * (ny + 1), M = (long long)nx * ny;
    if (MODE != 3 && col_ok && j0 >= 1) pb = v2[TOPO_IDX(c + rs * (j0 - 1), NN)];
    // Loads run two element rows ahead of their use (a strip is walked row by row, so one row of
    // lookahead leaves each row waiting for its own loads): *_n is used at the next iteration,
    // *_nn at the one after.  Element row e needs v of node row e + 1, x of element row e, and b,
    // the mask (and the FP64 residual for DOT 2) of node row e, the row it outputs.
    V2 pt_n = zero, pt_nn = zero, bb_n = zero, bb_nn = zero;
    T xe_n = T(0), xe_nn = T(0);
    uint16_t fx_n = 0, fx_nn = 0;
    double2 rr_n = make_double2(0.0, 0.0), rr_nn = make_double2(0.0, 0.0);
    {
      const int ey = j0 - 1;  // first iteration: element row j0 - 1, no output
      if (MODE != 3 && col_ok && ey + 1 <= ny) pt_n = v2[TOPO_IDX(c + rs * (ey + 1), NN)];
      if (el_col && ey >= 0 && ey < ny) xe_n = x[TOPO_IDX(c + nx * ey, M)];
      if (ey + 1 < j1) {  // second iteration: element row j0, output node row j0
        if (MODE != 3 && col_ok && ey + 2 <= ny) pt_nn = v2[TOPO_IDX(c + rs * (ey + 2), NN)];
        if (el_col && ey + 1 < ny) xe_nn = x[TOPO_IDX(c + nx * (ey + 1), M)];
        if (out_lane) {
          const int nn = TOPO_IDX(c + rs * (ey + 1), NN);
          fx_nn = *reinterpret_cast<const uint16_t*>(fixed + 2 * nn);
          if (MODE != 0) bb_nn = b2[nn];
          if (DOT == 2) rr_nn = reinterpret_cast<const double2*>(rdot)[nn];
        }
      }
    }
    T cu = T(0), cv = T(0), xcarry = T(0);
    for (int ey = j0 - 1; ey < j1; ++ey) {
      const V2 pt = pt_n;
      const T xe = xe_n;
      const V2 bb = bb_n;
      const uint16_t fx = fx_n;
      const double2 rr = rr_n;
      pt_n = pt_nn;
      xe_n = xe_nn;
      bb_n = bb_nn;
      fx_n = fx_nn;
      rr_n = rr_nn;
      pt_nn = zero;
      xe_nn = T(0);
      if (ey + 2 < j1) {  // loads of the iteration after next: element row ey + 2
        if (MODE != 3 && col_ok && ey + 3 <= ny) pt_nn = v2[TOPO_IDX(c + rs * (ey + 3), NN)];
        if (el_col && ey + 2 < ny) xe_nn = x[TOPO_IDX(c + nx * (ey + 2), M)];
        if (out_lane) {
          const int nn = TOPO_IDX(c + rs * (ey + 2), NN);
          fx_nn = *reinterpret_cast<const uint16_t*>(fixed + 2 * nn);
          if (MODE != 0) bb_nn = b2[nn];
          if (DOT == 2) rr_nn = reinterpret_cast<const double2*>(rdot)[nn];
        }
      }
      const T pbr_u = shfl_dn(pb.x), pbr_v = shfl_dn(pb.y);
      const T ptr_u = shfl_dn(pt.x), ptr_v = shfl_dn(pt.y);
      T ru[4], rv[4];
      if (MODE != 3) {
        const T uu[4] = {pb.x, pbr_u, ptr_u, pt.x};
        const T vv[4] = {pb.y, pbr_v, ptr_v, pt.y};
        q1_element<T>(k, xe, uu, vv, ru, rv);
      } else {
#pragma unroll
        for (int a = 0; a < 4; ++a) ru[a] = rv[a] = T(0);
      }
      const T l1u = shfl_up1(ru[1]), l1v = shfl_up1(rv[1]);
      const T l2u = shfl_up1(ru[2]), l2v = shfl_up1(rv[2]);
      const T xl = shfl_up1(xe);
      const T xpair = xe + (lane >= 1 ? xl : T(0));
      if (ey >= j0 && out_lane) {
        const T qu = cu + ru[0] + l1u, qv = cv + rv[0] + l1v;
        const int node = c + rs * ey;
        V2 out;
        if (MODE == 0) {
          out.x = qu;
          out.y = qv;
        } else if (MODE == 1) {
          out.x = bb.x - qu;
          out.y = bb.y - qv;
        } else {
          const T xs = xcarry + xpair;
          const T dinv = xs > T(0) ? recip_rn(k.kd * xs) : T(1);
          if (MODE == 2) {
            out.x = fma(omega * dinv, bb.x - qu, pb.x);
            out.y = fma(omega * dinv, bb.y - qv, pb.y);
          } else {
            out.x = omega * dinv * bb.x;
            out.y = omega * dinv * bb.y;
          }
        }
        if (fx & 0xff) out.x = T(0);
        if (fx >> 8) out.y = T(0);
        if (TOPO_IN(node, NN)) reinterpret_cast<V2*>(y)[node] = out;
        if (DOT == 1) part = fma(double_of(pb.x), double_of(out.x), fma(double_of(pb.y), double_of(out.y), part));
        if (DOT == 2) part = fma(rr.x, double_of(out.x), fma(rr.y, double_of(out.y), part));
      }
      cu = ru[3] + l2u;
      cv = rv[3] + l2v;
      xcarry = xpair;
      pb = pt;
    }
  }
  if (!DOT) return;
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

// ---- Residual and restriction in one pass --------------------------------------------------
// b_c = P^T (b - K(x) v) on the finest level: the residual rows of k_q1_sweep<T, 1, 0> (the same
// arithmetic), never stored, are combined into the coarse right-hand side by the 9-point full
// weighting in the order of k_restrict (per coarse node: fine rows 2J - 1, 2J, 2J + 1, and in
// each row the columns 2I - 1, 2I, 2I + 1), so the coarse values are the same bits as those of
// the two separate kernels.  A warp owns kRRCols coarse columns, I = kRRCols wc + 1 ..
// kRRCols (wc + 1) (and I = 0 in the first warp), and a strip of coarse rows; its lanes cover the
// fine columns 2 kRRCols wc - 1 .. 2 kRRCols wc + 30, residuals on lanes 1..30, so that each owned
// 3-column stencil lies on them, and it walks the fine rows 2 J0 - 1 .. 2 J1 - 1 (the row below
// the strip is recomputed).  Loads run two element rows ahead, as in k_q1_sweep.
constexpr int kRRCols = 14;

template <typename T>
__global__ void __launch_bounds__(kQ1Warps * 32) k_q1_resrestrict(int nx, int ny, int crows,
                                                                   Q1K<T> k,
                                                                   const T* __restrict__ x,
                                                                   const T* __restrict__ v,
                                                                   const T* __restrict__ b,
                                                                   T* __restrict__ bc,
                                                                   const uint8_t* __restrict__ fixed,
                                                                   const uint8_t* __restrict__ fixed_c,
                                                                   const CgScalars* sc) {
  pdl_prologue();
  using V2 = typename Vec2<T>::type;
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const long long n = 2LL * (nx + 1) * (ny + 1);
  const int cnx = nx / 2, cny = ny / 2;
  v += rhs * n;
  b += rhs * n;
  bc += rhs * 2LL * (cnx + 1) * (cny + 1);
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kQ1Warps + (threadIdx.x >> 5);
  const int ncolw = (cnx + kRRCols - 1) / kRRCols;
  const int nstrip = (cny + 1 + crows - 1) / crows;
  const int wc = gw % ncolw, ws = gw / ncolw;
  if (ws >= nstrip) return;
  const int c = wc * 2 * kRRCols - 1 + lane;  // fine node column and element column of the lane
  const bool col_ok = (c >= 0 && c <= nx);
  const bool out_lane = (lane >= 1 && lane <= 30 && col_ok);
  const bool el_col = (lane <= 30 && c >= 0 && c < nx);
  const bool own = col_ok && (c & 1) == 0 && ((lane >= 3 && lane <= 2 * kRRCols + 1) ||
                                              (wc == 0 && lane == 1));
  const int I = c >> 1;
  const int J0 = ws * crows, J1 = min(J0 + crows, cny + 1);
  const int j0 = max(2 * J0 - 1, 0), j1 = min(2 * J1 - 1, ny) + 1;  // fine rows [j0, j1)
  const V2* v2 = reinterpret_cast<const V2*>(v);
  const V2* b2 = reinterpret_cast<const V2*>(b);
  const int rs = nx + 1;
  V2 zero;
  zero.x = T(0);
  zero.y = T(0);
  V2 pb = zero;
  if (col_ok && j0 >= 1) pb = v2[c + rs * (j0 - 1)];
  V2 pt_n = zero, pt_nn = zero, bb_n = zero, bb_nn = zero;
  T xe_n = T(0), xe_nn = T(0);
  uint16_t fx_n = 0, fx_nn = 0;
  {
    const int ey = j0 - 1;
    if (col_ok && ey + 1 <= ny) pt_n = v2[c + rs * (ey + 1)];
    if (el_col && ey >= 0 && ey < ny) xe_n = x[c + nx * ey];
    if (ey + 1 < j1) {
      if (col_ok && ey + 2 <= ny) pt_nn = v2[c + rs * (ey + 2)];
      if (el_col && ey + 1 < ny) xe_nn = x[c + nx * (ey + 1)];
      if (out_lane) {
        const int nn = c + rs * (ey + 1);
        fx_nn = *reinterpret_cast<const uint16_t*>(fixed + 2 * nn);
        bb_nn = b2[nn];
      }
    }
  }
  T cu = T(0), cv = T(0);
  T ax = T(0), ay = T(0);  // the full-weighting sums of the coarse row in progress
  for (int ey = j0 - 1; ey < j1; ++ey) {
    const V2 pt = pt_n;
    const T xe = xe_n;
    const V2 bb = bb_n;
    const uint16_t fx = fx_n;
    pt_n = pt_nn;
    xe_n = xe_nn;
    bb_n = bb_nn;
    fx_n = fx_nn;
    pt_nn = zero;
    xe_nn = T(0);
    if (ey + 2 < j1) {
      if (col_ok && ey + 3 <= ny) pt_nn = v2[c + rs * (ey + 3)];
      if (el_col && ey + 2 < ny) xe_nn = x[c + nx * (ey + 2)];
      if (out_lane) {
        const int nn = c + rs * (ey + 2);
        fx_nn = *reinterpret_cast<const uint16_t*>(fixed + 2 * nn);
        bb_nn = b2[nn];
      }
    }
    const T pbr_u = shfl_dn(pb.x), pbr_v = shfl_dn(pb.y);
    const T ptr_u = shfl_dn(pt.x), ptr_v = shfl_dn(pt.y);
    T ru[4], rv[4];
    {
      const T uu[4] = {pb.x, pbr_u, ptr_u, pt.x};
      const T vv[4] = {pb.y, pbr_v, ptr_v, pt.y};
      q1_element<T>(k, xe, uu, vv, ru, rv);
    }
    const T l1u = shfl_up1(ru[1]), l1v = shfl_up1(rv[1]);
    const T l2u = shfl_up1(ru[2]), l2v = shfl_up1(rv[2]);
    if (ey >= j0) {  // residual of node row ey (warp-uniform), then its share of P^T r
      V2 r = zero;
      if (out_lane) {
        const T qu = cu + ru[0] + l1u, qv = cv + rv[0] + l1v;
        r.x = bb.x - qu;
        r.y = bb.y - qv;
        if (fx & 0xff) r.x = T(0);
        if (fx >> 8) r.y = T(0);
      }
      const T rlx = shfl_up1(r.x), rly = shfl_up1(r.y);
      const T rrx = shfl_dn(r.x), rry = shfl_dn(r.y);
      // one fine row of the weighting, with the row weight wy (k_restrict's order)
      auto row_terms = [&](T wy, T& sx, T& sy) {
        if (c - 1 >= 0) {
          const T w = wy * T(0.5);
          sx = fma(w, rlx, sx);
          sy = fma(w, rly, sy);
        }
        sx = fma(wy, r.x, sx);
        sy = fma(wy, r.y, sy);
        if (c + 1 <= nx) {
          const T w = wy * T(0.5);
          sx = fma(w, rrx, sx);
          sy = fma(w, rry, sy);
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
    cu = ru[3] + l2u;
    cv = rv[3] + l2v;
    pb = pt;
  }
}

// ---- Fused pairs of V-cycle steps on the finest level ----------------------------------------
// MODE 4: the first two damped-Jacobi sweeps from zero, z = omega D^{-1} b then
//         y = z + omega D^{-1} (b - K z), with z formed on the fly from b and x (no z pass).
// MODE 5: the prolongation and correction t + P zc followed by one sweep on the corrected
//         iterate, y = v + omega D^{-1} (b - K v) with v = t + P zc formed on the fly (zc: the
//         level-1 correction, (nx/2 + 1) x (ny/2 + 1) nodes).
// The per-node arithmetic and its order are those of k_q1_sweep (modes 3 and 2) and k_prolong_add,
// so the results are the same bits as the unfused steps.  Loads run one element row ahead.
template <typename T, int MODE>
__global__ void __launch_bounds__(kQ1Warps * 32) k_q1_fused(int nx, int ny, int rows, Q1K<T> k,
                                                             const T* __restrict__ x,
                                                             const T* __restrict__ t,
                                                             const T* __restrict__ zc,
                                                             const T* __restrict__ b,
                                                             T* __restrict__ y, T omega,
                                                             const uint8_t* __restrict__ fixed,
                                                             const CgScalars* sc) {
  static_assert(MODE == 4 || MODE == 5, "fused modes");
  pdl_prologue();
  using V2 = typename Vec2<T>::type;
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const long long n = 2LL * (nx + 1) * (ny + 1);
  const long long ncn = (long long)(nx / 2 + 1) * (ny / 2 + 1);
  b += rhs * n;
  y += rhs * n;
  if (MODE == 5) {
    t += rhs * n;
    zc += rhs * 2 * ncn;
  }
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kQ1Warps + (threadIdx.x >> 5);
  const int ncolw = (nx + 1 + kQ1Cols - 1) / kQ1Cols;
  const int nstrip = (ny + 1 + rows - 1) / rows;
  const int wc = gw % ncolw, ws = gw / ncolw;
  if (ws >= nstrip) return;
  const int c = wc * kQ1Cols - 1 + lane;
  const bool col_ok = (c >= 0 && c <= nx);
  const bool out_lane = (lane >= 1 && lane <= kQ1Cols && col_ok);
  const bool el_col = (lane <= kQ1Cols && c >= 0 && c < nx);
  // MODE 4 forms D^{-1} on every lane's node: every lane needs its own element column's density
  // and lane 0 also the one to its left (the other lanes get it by a shuffle)
  const bool xcol = MODE == 4 ? (c >= 0 && c < nx) : el_col;
  const bool xleft0 = MODE == 4 && lane == 0 && c - 1 >= 0 && c - 1 < nx;
  const int j0 = ws * rows;
  const int j1 = min(j0 + rows, ny + 1);
  const int rs = nx + 1;
  const int crs = nx / 2 + 1;
  const V2* b2 = reinterpret_cast<const V2*>(b);
  const V2* t2 = reinterpret_cast<const V2*>(t);
  const V2* zc2 = reinterpret_cast<const V2*>(zc);
  V2 zero;
  zero.x = T(0);
  zero.y = T(0);
  // raw data of node row r (element row r for the densities)
  struct Raw {
    V2 b, t, z00, z10, z01, z11;
    T xe, xl0;
    uint16_t fx;
  };
  auto load = [&](int r, Raw& R) {
    R.b = zero;
    R.t = zero;
    R.z00 = R.z10 = R.z01 = R.z11 = zero;
    R.xe = T(0);
    R.xl0 = T(0);
    R.fx = 0;
    if (r < 0 || r > ny) return;
    if (xcol && r < ny) R.xe = x[c + nx * r];
    if (xleft0 && r < ny) R.xl0 = x[c - 1 + nx * r];
    if (!col_ok) return;
    const int nd = c + rs * r;
    R.fx = *reinterpret_cast<const uint16_t*>(fixed + 2 * nd);
    R.b = b2[nd];
    if (MODE == 5) {
      R.t = t2[nd];
      const int i0 = c >> 1, i1 = (c + 1) >> 1, q0 = r >> 1, q1 = (r + 1) >> 1;
      R.z00 = zc2[i0 + crs * q0];
      R.z10 = zc2[i1 + crs * q0];
      R.z01 = zc2[i0 + crs * q1];
      R.z11 = zc2[i1 + crs * q1];
    }
  };
  // xpair(r) = x(c, r) + x(c - 1, r), the left density by a shuffle (lane 0: its own load)
  auto xpair_of = [&](const Raw& R) {
    const T xl = shfl_up1(R.xe);
    return R.xe + (lane >= 1 ? xl : (MODE == 4 ? R.xl0 : T(0)));
  };
  auto dinv_of = [&](T xs) { return xs > T(0) ? recip_rn(k.kd * xs) : T(1); };
  // the input node value v(r) of the sweep
  T dinv_in = T(0);  // MODE 4: the diagonal of the last input row, reused at its output
  auto input = [&](int r, const Raw& R, T xpair_prev, T xpair_r) {
    V2 v = zero;
    if (MODE == 4) {
      const T dinv = dinv_of(xpair_prev + xpair_r);
      dinv_in = dinv;
      v.x = mul_rn(mul_rn(omega, dinv), R.b.x);
      v.y = mul_rn(mul_rn(omega, dinv), R.b.y);
      if (R.fx & 0xff) v.x = T(0);
      if (R.fx >> 8) v.y = T(0);
    } else {
      const T wxh = (c & 1) ? T(0.5) : T(1);
      const T wyh = (r & 1) ? T(0.5) : T(1);
      const T w = wxh * wyh * T(1);
      T ax = T(0), ay = T(0);
      ax = fma(w, R.z00.x, ax);
      ay = fma(w, R.z00.y, ay);
      if (c & 1) {
        ax = fma(w, R.z10.x, ax);
        ay = fma(w, R.z10.y, ay);
      }
      if (r & 1) {
        ax = fma(w, R.z01.x, ax);
        ay = fma(w, R.z01.y, ay);
        if (c & 1) {
          ax = fma(w, R.z11.x, ax);
          ay = fma(w, R.z11.y, ay);
        }
      }
      v = R.t;
      if (!(R.fx & 0xff)) v.x = R.t.x + ax;
      if (!(R.fx >> 8)) v.y = R.t.y + ay;
    }
    return v;
  };
  // start: rows j0 - 2 (densities only), j0 - 1 (the first element row) and j0 (its top nodes)
  Raw Rm, Rc, Rn;
  load(j0 - 2, Rm);
  load(j0 - 1, Rc);
  load(j0, Rn);
  T xpair_m = xpair_of(Rm);
  if (j0 - 2 < 0) xpair_m = T(0);
  T xpair_c = xpair_of(Rc);
  V2 pb = (j0 - 1 >= 0 && col_ok) ? input(j0 - 1, Rc, xpair_m, xpair_c) : zero;
  T xcarry = T(0);
  T cu = T(0), cv = T(0);
  for (int ey = j0 - 1; ey < j1; ++ey) {
    const Raw R = Rc;   // node row ey: b, mask; element row ey: density
    const Raw N = Rn;   // node row ey + 1
    if (ey + 2 <= ny && ey + 1 < j1) load(ey + 2, Rn);
    else Rn = Raw{zero, zero, zero, zero, zero, zero, T(0), T(0), 0};
    Rc = N;
    const T dinv_row = dinv_in;  // (MODE 4: node row ey's, formed when it was the input row)
    const T xpair_n = xpair_of(N);
    const V2 pt = (ey + 1 <= ny && col_ok) ? input(ey + 1, N, xpair_c, xpair_n) : zero;
    const T xe = el_col ? R.xe : T(0);
    const T pbr_u = shfl_dn(pb.x), pbr_v = shfl_dn(pb.y);
    const T ptr_u = shfl_dn(pt.x), ptr_v = shfl_dn(pt.y);
    T ru[4], rv[4];
    {
      const T uu[4] = {pb.x, pbr_u, ptr_u, pt.x};
      const T vv[4] = {pb.y, pbr_v, ptr_v, pt.y};
      q1_element<T>(k, xe, uu, vv, ru, rv);
    }
    const T l1u = shfl_up1(ru[1]), l1v = shfl_up1(rv[1]);
    const T l2u = shfl_up1(ru[2]), l2v = shfl_up1(rv[2]);
    const T xl = shfl_up1(xe);
    const T xpair = xe + (lane >= 1 ? xl : T(0));
    if (ey >= j0 && out_lane) {
      const T qu = cu + ru[0] + l1u, qv = cv + rv[0] + l1v;
      const T dinv = MODE == 4 ? dinv_row : dinv_of(xcarry + xpair);
      V2 out;
      out.x = fma(omega * dinv, R.b.x - qu, pb.x);
      out.y = fma(omega * dinv, R.b.y - qv, pb.y);
      if (R.fx & 0xff) out.x = T(0);
      if (R.fx >> 8) out.y = T(0);
      reinterpret_cast<V2*>(y)[c + rs * ey] = out;
    }
    cu = ru[3] + l2u;
    cv = rv[3] + l2v;
    xcarry = xpair;
    xpair_c = xpair_n;
    pb = pt;
  }
}

// ---- Outer operator in pair-of-FP32 arithmetic ------------------------------------------------
// GB300 issues about 2 FP64 operations per clock per SM against 128 FP32 ones, so the FP64 outer
// operator of the mixed solver is ALU-bound at ~40 FP64 operations per element.  This variant
// computes the same butterfly with each value held as an unevaluated sum hi + lo of two floats
// (Dekker's double-float arithmetic with error-free TwoSum and FMA-based TwoProd, about 48
// significant bits): p is split into float pairs with integer operations, q is rebuilt as
// double(hi) + double(lo) (one FP64 add per DOF), and p^T q is accumulated in pairs.  Values
// below 2^-100 in magnitude lose their low part (float range); 48 bits keep the CG recurrences of
// the mixed solver far below its 1e-8 tolerance.  All adds and multiplies use the _rn intrinsics
// so that the compiler cannot contract them into fused operations that break the error terms.
struct Q1KD {
  f2 c11, c12, c22, c33, cH, cHp;
};

// The butterfly of q1_element in pair arithmetic (the density applied after Khat).
__device__ __forceinline__ void q1_element_df(const Q1KD& k, f2 xe, const f2 u[4], const f2 v[4],
                                              f2 ru[4], f2 rv[4]) {
  const f2 d1 = df_sub_nr(u[2], u[0]), d2 = df_sub_nr(u[1], u[3]);
  const f2 s1 = df_add_nr(u[0], u[2]), s2 = df_add_nr(u[1], u[3]);
  const f2 X = df_add_nr(d2, d1), Y = df_sub_nr(d1, d2), H = df_sub_nr(s1, s2);
  const f2 e1 = df_sub_nr(v[2], v[0]), e2 = df_sub_nr(v[1], v[3]);
  const f2 t1 = df_add_nr(v[0], v[2]), t2 = df_add_nr(v[1], v[3]);
  const f2 Xp = df_add_nr(e2, e1), Yp = df_sub_nr(e1, e2), Hp = df_sub_nr(t1, t2);
  const f2 G = df_add_nr(Y, Xp);
  const f2 gX = df_mul_nr(xe, df_add_nr(df_mul_nr(k.c11, X), df_mul_nr(k.c12, Yp)));
  const f2 gYp = df_mul_nr(xe, df_add_nr(df_mul_nr(k.c12, X), df_mul_nr(k.c22, Yp)));
  const f2 gG = df_mul_nr(xe, df_mul_nr(k.c33, G));
  const f2 gH = df_mul_nr(xe, df_mul_nr(k.cH, H));
  const f2 gHp = df_mul_nr(xe, df_mul_nr(k.cHp, Hp));
  const f2 A = df_add_nr(gX, gG), B = df_sub_nr(gX, gG);
  ru[0] = df_sub_nr(gH, A);
  ru[1] = df_sub_nr(B, gH);
  ru[2] = df_add_nr(A, gH);
  ru[3] = df_sub_nr(df_neg(B), gH);
  const f2 C = df_add_nr(gYp, gG), Dd = df_sub_nr(gYp, gG);
  rv[0] = df_sub_nr(gHp, C);
  rv[1] = df_sub_nr(df_neg(Dd), gHp);
  rv[2] = df_add_nr(C, gHp);
  rv[3] = df_sub_nr(Dd, gHp);
}

__device__ __forceinline__ f2 shfl_dn_df(f2 a) { return {shfl_dn(a.h), shfl_dn(a.l)}; }
__device__ __forceinline__ f2 shfl_up1_df(f2 a) { return {shfl_up1(a.h), shfl_up1(a.l)}; }

// q = K(x) p with p^T q and alpha (as k_q1_sweep<double, 0, 1>), in pair arithmetic.  xdf: the
// densities as float pairs.
__global__ void __launch_bounds__(kQ1Warps * 32) k_q1_sweep_df(int nx, int ny, int rows, Q1KD k,
                                                                const float2* __restrict__ xdf,
                                                                const double* __restrict__ v,
                                                                double* __restrict__ y,
                                                                const uint8_t* __restrict__ fixed,
                                                                CgScalars* sc, double* partials,
                                                                unsigned* counters) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const long long n = 2LL * (nx + 1) * (ny + 1);
  v += rhs * n;
  y += rhs * n;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kQ1Warps + (threadIdx.x >> 5);
  const int ncolw = (nx + 1 + kQ1Cols - 1) / kQ1Cols;
  const int nstrip = (ny + 1 + rows - 1) / rows;
  const int wc = gw % ncolw, ws = gw / ncolw;
  f2 part = {0.0f, 0.0f};
  if (ws < nstrip) {
    const int c = wc * kQ1Cols - 1 + lane;
    const bool col_ok = (c >= 0 && c <= nx);
    const bool out_lane = (lane >= 1 && lane <= kQ1Cols && col_ok);
    const bool el_col = (lane <= kQ1Cols && c >= 0 && c < nx);
    const int j0 = ws * rows;
    const int j1 = min(j0 + rows, ny + 1);
    const double2* v2 = reinterpret_cast<const double2*>(v);
    const int rs = nx + 1;
    const f2 z = {0.0f, 0.0f};
    f2 pbu = z, pbv = z;
    if (col_ok && j0 >= 1) {
      const double2 t = v2[c + rs * (j0 - 1)];
      pbu = df_from_double(t.x);
      pbv = df_from_double(t.y);
    }
    // two element rows of lookahead, as in k_q1_sweep
    double2 pt_n = make_double2(0.0, 0.0), pt_nn = make_double2(0.0, 0.0);
    float2 xe_n = make_float2(0.0f, 0.0f), xe_nn = make_float2(0.0f, 0.0f);
    uint16_t fx_n = 0, fx_nn = 0;
    {
      const int ey = j0 - 1;
      if (col_ok && ey + 1 <= ny) pt_n = v2[c + rs * (ey + 1)];
      if (el_col && ey >= 0 && ey < ny) xe_n = xdf[c + nx * ey];
      if (ey + 1 < j1) {
        if (col_ok && ey + 2 <= ny) pt_nn = v2[c + rs * (ey + 2)];
        if (el_col && ey + 1 < ny) xe_nn = xdf[c + nx * (ey + 1)];
        if (out_lane) fx_nn = *reinterpret_cast<const uint16_t*>(fixed + 2 * (c + rs * (ey + 1)));
      }
    }
    f2 cu = z, cv = z;
    for (int ey = j0 - 1; ey < j1; ++ey) {
      const f2 ptu = df_from_double(pt_n.x), ptv = df_from_double(pt_n.y);
      const f2 xe = {xe_n.x, xe_n.y};
      const uint16_t fx = fx_n;
      pt_n = pt_nn;
      xe_n = xe_nn;
      fx_n = fx_nn;
      pt_nn = make_double2(0.0, 0.0);
      xe_nn = make_float2(0.0f, 0.0f);
      if (ey + 2 < j1) {
        if (col_ok && ey + 3 <= ny) pt_nn = v2[c + rs * (ey + 3)];
        if (el_col && ey + 2 < ny) xe_nn = xdf[c + nx * (ey + 2)];
        if (out_lane) fx_nn = *reinterpret_cast<const uint16_t*>(fixed + 2 * (c + rs * (ey + 2)));
      }
      const f2 uu[4] = {pbu, shfl_dn_df(pbu), shfl_dn_df(ptu), ptu};
      const f2 vv[4] = {pbv, shfl_dn_df(pbv), shfl_dn_df(ptv), ptv};
      f2 ru[4], rv[4];
      q1_element_df(k, xe, uu, vv, ru, rv);
      const f2 l1u = shfl_up1_df(ru[1]), l1v = shfl_up1_df(rv[1]);
      const f2 l2u = shfl_up1_df(ru[2]), l2v = shfl_up1_df(rv[2]);
      if (ey >= j0 && out_lane) {
        f2 qu = df_add_nr(df_add_nr(cu, ru[0]), l1u), qv = df_add_nr(df_add_nr(cv, rv[0]), l1v);
        if (fx & 0xff) qu = z;
        if (fx >> 8) qv = z;
        double2 out;
        out.x = double_from_float(qu.h) + double_from_float(qu.l);
        out.y = double_from_float(qv.h) + double_from_float(qv.l);
        reinterpret_cast<double2*>(y)[c + rs * ey] = out;
        part = df_add(part, df_add(df_mul(pbu, qu), df_mul(pbv, qv)));
      }
      cu = df_add_nr(ru[3], l2u);
      cv = df_add_nr(rv[3], l2v);
      pbu = ptu;
      pbv = ptv;
    }
  }
  const double bs = block_sum_q1(double_from_float(part.h) + double_from_float(part.l));
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

// The densities checked (flag set if one is not finite and > 0) and converted for the FP32
// V-cycle (x32) and the pair-arithmetic operator (xdf) in one pass; x32, xdf may be null.
__global__ void k_prepare_x(const double* __restrict__ x, long long m, int* flag,
                            float* __restrict__ x32, float2* __restrict__ xdf) {
  pdl_prologue();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double v = x[i];
  if (!(v > 0.0) || !isfinite(v)) *flag = 1;
  if (x32) x32[i] = (float)v;
  if (xdf) {
    const f2 t = df_from_double(v);
    xdf[i] = make_float2(t.h, t.l);
  }
}

// Densities as float pairs (hi + lo) for k_q1_sweep_df.
__global__ void k_split_df(const double* __restrict__ x, float2* __restrict__ out, long long m) {
  pdl_prologue();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    const f2 t = df_from_double(x[i]);
    out[i] = make_float2(t.h, t.l);
  }
}

// First coarse level, matrix-free Galerkin operator A_1 = P^T K(x) P applied element by element:
// the coarse element's four nodal values are interpolated bilinearly to the 3 x 3 fine nodes of
// its four children, each child's x_c K0 is applied in the butterfly form, and the 3 x 3 fine
// forces are restricted back to the four coarse nodes (weights 1, 1/2, 1/4).  Same warp-sweep
// data movement as k_q1_sweep on the coarse grid (nx, ny = coarse elements); xf holds the finest
// densities (2nx x 2ny), invd the level's inverse diagonal (modes 2, 3).
// MODE 4 and 5 fuse pairs of steps as k_q1_fused does on the finest level: 4 = the first two sweeps
// from zero (z = omega invd b formed on the fly), 5 = the prolongation and correction t + P zc
// (zc: the second coarse level's vector) formed on the fly, then one sweep; the same bits as the
// separate steps.
template <int MODE>
__global__ void __launch_bounds__(kQ1Warps * 32) k_q1g_sweep(int nx, int ny, int rows,
                                                              Q1K<float> k,
                                                              const float* __restrict__ xf,
                                                              const float* __restrict__ v,
                                                              const float* __restrict__ b,
                                                              float* __restrict__ y, float omega,
                                                              const float* __restrict__ invd,
                                                              const uint8_t* __restrict__ fixed,
                                                              const CgScalars* sc,
                                                              const float* __restrict__ zc) {
  constexpr bool FUSED = MODE == 4 || MODE == 5;
  constexpr bool SWEEP = MODE == 2 || FUSED;  // output y = v + omega invd (b - A v)
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const long long n = 2LL * (nx + 1) * (ny + 1);
  const long long ncn = (long long)(nx / 2 + 1) * (ny / 2 + 1);
  v += rhs * n;
  y += rhs * n;
  b += rhs * n;
  if (MODE == 5) zc += rhs * 2 * ncn;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kQ1Warps + (threadIdx.x >> 5);
  const int ncolw = (nx + 1 + kQ1Cols - 1) / kQ1Cols;
  const int nstrip = (ny + 1 + rows - 1) / rows;
  const int wc = gw % ncolw, ws = gw / ncolw;
  if (ws >= nstrip) return;
  const int c = wc * kQ1Cols - 1 + lane;
  const bool col_ok = (c >= 0 && c <= nx);
  const bool out_lane = (lane >= 1 && lane <= kQ1Cols && col_ok);
  const bool el_col = (lane <= kQ1Cols && c >= 0 && c < nx);
  const int j0 = ws * rows;
  const int j1 = min(j0 + rows, ny + 1);
  const int fnx = 2 * nx;
  const int rs = nx + 1;
  const int crs = nx / 2 + 1;
  const float2* v2 = reinterpret_cast<const float2*>(v);
  const float2* zc2 = reinterpret_cast<const float2*>(zc);
  const float2 z2 = make_float2(0.f, 0.f);
  // the fused modes form the swept vector on every lane's node (node data of all rows)
  const bool node_data = FUSED ? col_ok : out_lane;
  // Two element rows of lookahead (see k_q1_sweep): iteration e reads v of node row e + 1 (the
  // stored iterate; MODE 5: t and the four zc values around node row e + 1), the four child
  // densities of coarse element row e, and b, invd and the mask of node row e.
  struct Raw {
    float2 pt, xb, xt, bb, di, z00, z10, z01, z11;
    uint16_t fx;
  };
  auto load_row = [&](int e, Raw& R) {
    R.pt = R.xb = R.xt = R.bb = R.di = z2;
    R.fx = 0;
    R.z00 = R.z10 = R.z01 = R.z11 = z2;
    if (MODE != 3 && MODE != 4 && col_ok && e + 1 <= ny) R.pt = v2[c + rs * (e + 1)];
    if (MODE == 5 && col_ok && e + 1 <= ny) {
      const int r = e + 1, i0 = c >> 1, i1 = (c + 1) >> 1, q0 = r >> 1, q1 = (r + 1) >> 1;
      R.z00 = zc2[i0 + crs * q0];
      R.z10 = zc2[i1 + crs * q0];
      R.z01 = zc2[i0 + crs * q1];
      R.z11 = zc2[i1 + crs * q1];
    }
    if (MODE != 3 && el_col && e >= 0 && e < ny) {
      R.xb = *reinterpret_cast<const float2*>(xf + 2 * c + fnx * (2 * e));
      R.xt = *reinterpret_cast<const float2*>(xf + 2 * c + fnx * (2 * e + 1));
    }
    if (e >= (FUSED ? 0 : j0) && e <= ny && node_data) {
      const int node = c + rs * e;
      R.fx = *reinterpret_cast<const uint16_t*>(fixed + 2 * node);
      if (MODE != 0) R.bb = reinterpret_cast<const float2*>(b)[node];
      if (MODE != 0 && MODE != 1) R.di = reinterpret_cast<const float2*>(invd)[node];
    }
  };
  // the swept vector at node row r of this lane: MODE 4 from the row's own b, invd and mask (as
  // MODE 3 writes it), MODE 5 from t (tv) and the zc values around the node (as k_prolong_add)
  auto fused_input = [&](int r, float2 tv, const Raw& nodeR, const Raw& zR) {
    float2 out = z2;
    if (MODE == 4) {
      out.x = mul_rn(mul_rn(omega, nodeR.di.x), nodeR.bb.x);
      out.y = mul_rn(mul_rn(omega, nodeR.di.y), nodeR.bb.y);
      if (nodeR.fx & 0xff) out.x = 0.f;
      if (nodeR.fx >> 8) out.y = 0.f;
    } else if (MODE == 5) {
      const float wxh = (c & 1) ? 0.5f : 1.f;
      const float wyh = (r & 1) ? 0.5f : 1.f;
      const float w = wxh * wyh * 1.f;
      float ax = 0.f, ay = 0.f;
      ax = fmaf(w, zR.z00.x, ax);
      ay = fmaf(w, zR.z00.y, ay);
      if (c & 1) {
        ax = fmaf(w, zR.z10.x, ax);
        ay = fmaf(w, zR.z10.y, ay);
      }
      if (r & 1) {
        ax = fmaf(w, zR.z01.x, ax);
        ay = fmaf(w, zR.z01.y, ay);
        if (c & 1) {
          ax = fmaf(w, zR.z11.x, ax);
          ay = fmaf(w, zR.z11.y, ay);
        }
      }
      out = tv;
      if (!(nodeR.fx & 0xff)) out.x = tv.x + ax;
      if (!(nodeR.fx >> 8)) out.y = tv.y + ay;
    }
    return out;
  };
  Raw Rn{}, Rnn{};
  load_row(j0 - 1, Rn);
  if (j0 < j1 || FUSED) load_row(j0, Rnn);
  float2 pb = z2;
  if (MODE != 3 && MODE != 4 && col_ok && j0 >= 1) pb = v2[c + rs * (j0 - 1)];
  if (FUSED && col_ok && j0 >= 1) {
    Raw Rm{};
    load_row(j0 - 2, Rm);  // MODE 5: zc around node row j0 - 1
    pb = fused_input(j0 - 1, pb, Rn, Rm);
  }
  float cu = 0.f, cv = 0.f;
  for (int ey = j0 - 1; ey < j1; ++ey) {
    const Raw Cur = Rn;  // iteration ey: t of node row ey + 1, densities of row ey, node row ey
    Rn = Rnn;            // iteration ey + 1: node row ey + 1
    // the fused modes read the node data of row ey + 1 from the item of iteration ey + 1, so the
    // item of iteration j1 (node row j1, the top of the strip) is loaded too
    if (ey + 2 < j1 || (FUSED && ey + 2 == j1)) load_row(ey + 2, Rnn);
    const float2 xb = Cur.xb, xt = Cur.xt, bb = Cur.bb, di = Cur.di;
    const uint16_t fx = Cur.fx;
    float2 pt = Cur.pt;
    if (FUSED) pt = (col_ok && ey + 1 <= ny) ? fused_input(ey + 1, Cur.pt, Rn, Cur) : z2;
    const float pbr_u = shfl_dn(pb.x), pbr_v = shfl_dn(pb.y);
    const float ptr_u = shfl_dn(pt.x), ptr_v = shfl_dn(pt.y);
    float R[4][2] = {};  // coarse local nodes (0,0) (1,0) (1,1) (0,1), components u, v
    if (MODE != 3) {
      // fine nodal values on the 3 x 3 grid F[i][j] (i along x, j along y), by interpolation
      float fu[3][3], fv[3][3];
      fu[0][0] = pb.x; fu[2][0] = pbr_u; fu[2][2] = ptr_u; fu[0][2] = pt.x;
      fv[0][0] = pb.y; fv[2][0] = pbr_v; fv[2][2] = ptr_v; fv[0][2] = pt.y;
      fu[1][0] = 0.5f * (fu[0][0] + fu[2][0]); fv[1][0] = 0.5f * (fv[0][0] + fv[2][0]);
      fu[1][2] = 0.5f * (fu[0][2] + fu[2][2]); fv[1][2] = 0.5f * (fv[0][2] + fv[2][2]);
      fu[0][1] = 0.5f * (fu[0][0] + fu[0][2]); fv[0][1] = 0.5f * (fv[0][0] + fv[0][2]);
      fu[2][1] = 0.5f * (fu[2][0] + fu[2][2]); fv[2][1] = 0.5f * (fv[2][0] + fv[2][2]);
      fu[1][1] = 0.5f * (fu[1][0] + fu[1][2]); fv[1][1] = 0.5f * (fv[1][0] + fv[1][2]);
      float Fu[3][3] = {}, Fv[3][3] = {};
      const float xc[2][2] = {{xb.x, xt.x}, {xb.y, xt.y}};  // [cx][cy]
#pragma unroll
      for (int cy = 0; cy < 2; ++cy)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
          const float uu[4] = {fu[cx][cy], fu[cx + 1][cy], fu[cx + 1][cy + 1], fu[cx][cy + 1]};
          const float vv[4] = {fv[cx][cy], fv[cx + 1][cy], fv[cx + 1][cy + 1], fv[cx][cy + 1]};
          float ru[4], rv[4];
          q1_element<float>(k, xc[cx][cy], uu, vv, ru, rv);
          Fu[cx][cy] += ru[0]; Fv[cx][cy] += rv[0];
          Fu[cx + 1][cy] += ru[1]; Fv[cx + 1][cy] += rv[1];
          Fu[cx + 1][cy + 1] += ru[2]; Fv[cx + 1][cy + 1] += rv[2];
          Fu[cx][cy + 1] += ru[3]; Fv[cx][cy + 1] += rv[3];
        }
      // restriction to the coarse corners: weight 1 at the corner, 1/2 on its two edges' midpoints,
      // 1/4 at the centre
      const int cxs[4] = {0, 2, 2, 0}, cys[4] = {0, 0, 2, 2};
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int i = cxs[a], j = cys[a];
        R[a][0] = Fu[i][j] + 0.5f * (Fu[1][j] + Fu[i][1]) + 0.25f * Fu[1][1];
        R[a][1] = Fv[i][j] + 0.5f * (Fv[1][j] + Fv[i][1]) + 0.25f * Fv[1][1];
      }
    }
    const float l1u = shfl_up1(R[1][0]), l1v = shfl_up1(R[1][1]);
    const float l2u = shfl_up1(R[2][0]), l2v = shfl_up1(R[2][1]);
    if (ey >= j0 && out_lane) {
      const float qu = cu + R[0][0] + l1u, qv = cv + R[0][1] + l1v;
      const int node = c + rs * ey;
      float2 out;
      if (MODE == 0) {
        out.x = qu;
        out.y = qv;
      } else {
        if (MODE == 1) {
          out.x = bb.x - qu;
          out.y = bb.y - qv;
        } else {
          if (SWEEP) {
            out.x = fmaf(omega * di.x, bb.x - qu, pb.x);
            out.y = fmaf(omega * di.y, bb.y - qv, pb.y);
          } else {
            out.x = omega * di.x * bb.x;
            out.y = omega * di.y * bb.y;
          }
        }
      }
      if (fx & 0xff) out.x = 0.f;
      if (fx >> 8) out.y = 0.f;
      reinterpret_cast<float2*>(y)[node] = out;
    }
    cu = R[3][0] + l2u;
    cv = R[3][1] + l2v;
    pb = pt;
  }
}

// Strip height: short enough that the grid has about one full wave of warps (152 SMs x 32),
// long enough to amortise the recomputed first element row of each strip.
int q1_rows(int nx, int ny) {
  const long long ncolw = (nx + 1 + kQ1Cols - 1) / kQ1Cols;
  const long long target = 152LL * 32;
  long long r = (ncolw * (ny + 1) + target - 1) / target;
  if (r < 2) r = 2;
  if (r > kQ1MaxRows) r = kQ1MaxRows;
  return (int)r;
}

unsigned q1_blocks(int nx, int ny) {
  const int rows = q1_rows(nx, ny);
  const long long warps = (long long)((nx + 1 + kQ1Cols - 1) / kQ1Cols) *
                          ((ny + 1 + rows - 1) / rows);
  return (unsigned)((warps + kQ1Warps - 1) / kQ1Warps);
}

}  // namespace

long long q1_partial_blocks(int nx, int ny) { return q1_blocks(nx, ny); }

template <typename T>
cudaError_t launch_q1_apply(int nx, int ny, int mode, const Q1Coef& coef, const T* x, const T* v,
                            const T* b, T* y, T omega, const uint8_t* fixed, int nrhs,
                            const CgScalars* sc, cudaStream_t st) {
  dim3 grid(q1_blocks(nx, ny), nrhs);
  const Q1K<T> k = coef_cast<T>(coef);
  CgScalars* scm = const_cast<CgScalars*>(sc);
  switch (mode) {
    case 0:
      topo::launch(k_q1_sweep<T, 0, 0>, grid, kQ1Warps * 32, 0, st, nx, ny, q1_rows(nx, ny), k, x, v, b, y, omega, fixed,
                                                               scm, nullptr, nullptr, nullptr);
      break;
    case 1:
      topo::launch(k_q1_sweep<T, 1, 0>, grid, kQ1Warps * 32, 0, st, nx, ny, q1_rows(nx, ny), k, x, v, b, y, omega, fixed,
                                                               scm, nullptr, nullptr, nullptr);
      break;
    case 2:
      topo::launch(k_q1_sweep<T, 2, 0>, grid, kQ1Warps * 32, 0, st, nx, ny, q1_rows(nx, ny), k, x, v, b, y, omega, fixed,
                                                               scm, nullptr, nullptr, nullptr);
      break;
    default:
      topo::launch(k_q1_sweep<T, 3, 0>, grid, kQ1Warps * 32, 0, st, nx, ny, q1_rows(nx, ny), k, x, v, b, y, omega, fixed,
                                                               scm, nullptr, nullptr, nullptr);
  }
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_q1_resrestrict(int nx, int ny, const Q1Coef& coef, const T* x, const T* v,
                                  const T* b, T* bc, const uint8_t* fixed,
                                  const uint8_t* fixed_c, int nrhs, const CgScalars* sc,
                                  cudaStream_t st) {
  const int cnx = nx / 2, cny = ny / 2;
  const long long ncolw = (cnx + kRRCols - 1) / kRRCols;
  const long long target = 152LL * 32;  // warps for about one per SM scheduler slot
  long long crows = (ncolw * (cny + 1) + target - 1) / target;
  if (crows < 1) crows = 1;
  if (crows > kQ1MaxRows / 2) crows = kQ1MaxRows / 2;
  const long long warps = ncolw * ((cny + 1 + crows - 1) / crows);
  dim3 grid((unsigned)((warps + kQ1Warps - 1) / kQ1Warps), nrhs);
  topo::launch(k_q1_resrestrict<T>, grid, kQ1Warps * 32, 0, st, nx, ny, (int)crows,
               coef_cast<T>(coef), x, v, b, bc, fixed, fixed_c, sc);
  return cudaGetLastError();
}
template cudaError_t launch_q1_resrestrict<double>(int, int, const Q1Coef&, const double*,
                                                   const double*, const double*, double*,
                                                   const uint8_t*, const uint8_t*, int,
                                                   const CgScalars*, cudaStream_t);
template cudaError_t launch_q1_resrestrict<float>(int, int, const Q1Coef&, const float*,
                                                  const float*, const float*, float*,
                                                  const uint8_t*, const uint8_t*, int,
                                                  const CgScalars*, cudaStream_t);

template cudaError_t launch_q1_apply<double>(int, int, int, const Q1Coef&, const double*,
                                             const double*, const double*, double*, double,
                                             const uint8_t*, int, const CgScalars*, cudaStream_t);
template cudaError_t launch_q1_apply<float>(int, int, int, const Q1Coef&, const float*,
                                            const float*, const float*, float*, float,
                                            const uint8_t*, int, const CgScalars*, cudaStream_t);

cudaError_t launch_q1g_apply(int nx, int ny, int mode, const Q1Coef& coef, const float* xf,
                             const float* v, const float* b, float* y, float omega,
                             const float* invd, const uint8_t* fixed, int nrhs,
                             const CgScalars* sc, cudaStream_t st, const float* zc) {
  dim3 grid(q1_blocks(nx, ny), nrhs);
  const Q1K<float> k = coef_cast<float>(coef);
  const int rows = q1_rows(nx, ny);
  switch (mode) {
    case 0:
      topo::launch(k_q1g_sweep<0>, grid, kQ1Warps * 32, 0, st, nx, ny, rows, k, xf, v, b, y, omega, invd, fixed, sc, zc);
      break;
    case 1:
      topo::launch(k_q1g_sweep<1>, grid, kQ1Warps * 32, 0, st, nx, ny, rows, k, xf, v, b, y, omega, invd, fixed, sc, zc);
      break;
    case 2:
      topo::launch(k_q1g_sweep<2>, grid, kQ1Warps * 32, 0, st, nx, ny, rows, k, xf, v, b, y, omega, invd, fixed, sc, zc);
      break;
    case 4:
      topo::launch(k_q1g_sweep<4>, grid, kQ1Warps * 32, 0, st, nx, ny, rows, k, xf, v, b, y, omega, invd, fixed, sc, zc);
      break;
    case 5:
      topo::launch(k_q1g_sweep<5>, grid, kQ1Warps * 32, 0, st, nx, ny, rows, k, xf, v, b, y, omega, invd, fixed, sc, zc);
      break;
    default:
      topo::launch(k_q1g_sweep<3>, grid, kQ1Warps * 32, 0, st, nx, ny, rows, k, xf, v, b, y, omega, invd, fixed, sc, zc);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_q1_smooth_beta(int nx, int ny, const Q1Coef& coef, const T* x, const T* v,
                                  const T* b, T* y, T omega, const uint8_t* fixed, int nrhs,
                                  const double* r, double* partials, unsigned* counters,
                                  CgScalars* sc, cudaStream_t st) {
  dim3 grid(q1_blocks(nx, ny), nrhs);
  topo::launch(k_q1_sweep<T, 2, 2>, grid, kQ1Warps * 32, 0, st, nx, ny, q1_rows(nx, ny), coef_cast<T>(coef),
                                                      x, v, b, y, omega, fixed, sc, partials,
                                                      counters, r);
  return cudaGetLastError();
}
template cudaError_t launch_q1_smooth_beta<double>(int, int, const Q1Coef&, const double*,
                                                   const double*, const double*, double*, double,
                                                   const uint8_t*, int, const double*, double*,
                                                   unsigned*, CgScalars*, cudaStream_t);
template cudaError_t launch_q1_smooth_beta<float>(int, int, const Q1Coef&, const float*,
                                                  const float*, const float*, float*, float,
                                                  const uint8_t*, int, const double*, double*,
                                                  unsigned*, CgScalars*, cudaStream_t);

template <typename T>
cudaError_t launch_q1_fused(int nx, int ny, int mode, const Q1Coef& coef, const T* x, const T* t,
                            const T* zc, const T* b, T* y, T omega, const uint8_t* fixed,
                            int nrhs, const CgScalars* sc, cudaStream_t st) {
  dim3 grid(q1_blocks(nx, ny), nrhs);
  const Q1K<T> k = coef_cast<T>(coef);
  if (mode == 4)
    topo::launch(k_q1_fused<T, 4>, grid, kQ1Warps * 32, 0, st, nx, ny, q1_rows(nx, ny), k, x, t,
                 zc, b, y, omega, fixed, sc);
  else
    topo::launch(k_q1_fused<T, 5>, grid, kQ1Warps * 32, 0, st, nx, ny, q1_rows(nx, ny), k, x, t,
                 zc, b, y, omega, fixed, sc);
  return cudaGetLastError();
}
template cudaError_t launch_q1_fused<double>(int, int, int, const Q1Coef&, const double*,
                                             const double*, const double*, const double*, double*,
                                             double, const uint8_t*, int, const CgScalars*,
                                             cudaStream_t);
template cudaError_t launch_q1_fused<float>(int, int, int, const Q1Coef&, const float*,
                                            const float*, const float*, const float*, float*,
                                            float, const uint8_t*, int, const CgScalars*,
                                            cudaStream_t);


cudaError_t launch_q1_apply_dot_df(int nx, int ny, const Q1Coef& coef, const float2* xdf,
                                   const double* v, double* y, const uint8_t* fixed, int nrhs,
                                   double* partials, unsigned* counters, CgScalars* sc,
                                   cudaStream_t st) {
  const Q1KD k{df_const(coef.c11), df_const(coef.c12), df_const(coef.c22), df_const(coef.c33),
               df_const(coef.cH), df_const(coef.cHp)};
  dim3 grid(q1_blocks(nx, ny), nrhs);
  topo::launch(k_q1_sweep_df, grid, kQ1Warps * 32, 0, st, nx, ny, q1_rows(nx, ny), k, xdf, v, y,
               fixed, sc, partials, counters);
  return cudaGetLastError();
}

cudaError_t launch_prepare_x(const double* x, long long m, int* flag, float* x32, float2* xdf,
                             cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  topo::launch(k_prepare_x, blocks_for(m), kThreads, 0, st, x, m, flag, x32, xdf);
  return cudaGetLastError();
}

cudaError_t launch_split_df(const double* x, float2* out, long long m, cudaStream_t st) {
  topo::launch(k_split_df, blocks_for(m), kThreads, 0, st, x, out, m);
  return cudaGetLastError();
}

cudaError_t launch_q1_apply_dot(int nx, int ny, const Q1Coef& coef, const double* x,
                                const double* v, double* y, const uint8_t* fixed, int nrhs,
                                double* partials, unsigned* counters, CgScalars* sc,
                                cudaStream_t st) {
  dim3 grid(q1_blocks(nx, ny), nrhs);
  topo::launch(k_q1_sweep<double, 0, 1>, grid, kQ1Warps * 32, 0, st, 
      nx, ny, q1_rows(nx, ny), coef_cast<double>(coef), x, v, nullptr, y, 0.0, fixed, sc, partials,
      counters, nullptr);
  return cudaGetLastError();
}

}  // namespace topo
