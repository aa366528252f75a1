// Host side of the MGCG library: solver objects, the Galerkin hierarchy, the V-cycle (Algorithm
// MG, Sec. 5.1) and the preconditioned CG loop (Algorithm PCG, Sec. 5.2) driven through CUDA
// graphs, and the C ABI of include/topo.h.
//
// The library runs on a private non-blocking stream.  Each call orders itself after the caller's
// stream (topo_set_stream, default the legacy stream) with an event and makes the caller's stream
// wait for its work on exit, so device pointers from the caller may be used on either side.
// A block of CG iterations is captured once per solver into a CUDA graph that the host replays,
// reading the scalars back once per block.  The kernels of a right-hand side whose recurrence has
// stopped return at once.  With topo_set_graph_mode(s, 1) one iteration is instead the body of a
// conditional while node, and a one-thread kernel at the end of the body clears the condition when
// every right-hand side has stopped: a whole solve is then one graph launch and one read-back.
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <type_traits>
#include <utility>
#include <string>
#include <vector>

#include "solver.cuh"

namespace topo {

thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

// TOPO_PDL=1 in the environment launches with programmatic dependent launch.  Off by default: on
// the 2048 x 1024 solve it measured 5% slower (dependent blocks waiting on the SMs).
bool pdl_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("TOPO_PDL");
    return v && v[0] == '1';
  }();
  return on;
}

topo_status cuda_status(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? TOPO_E_OOM : TOPO_E_CUDA;
}

// ---- Index-check records (debug build) ------------------------------------------------------
struct BoundsReg {
  BoundsReader reader;
  const char* file;
};
std::vector<BoundsReg>& bounds_readers() {
  static std::vector<BoundsReg> r;
  return r;
}

#ifdef TOPO_BOUNDS_CHECK
__global__ void k_bounds_selftest(long long i, long long n, int* out) {
  out[0] = TOPO_IN(i, n) ? 1 : 0;
}
#endif

// Sum of the records of every translation unit; the first nonzero one in *first.
cudaError_t read_bounds(unsigned long long* count, BoundsRecord* first, const char** file,
                        bool reset) {
  *count = 0;
  *first = BoundsRecord{};
  *file = "";
  cudaError_t e = cudaDeviceSynchronize();
  for (const BoundsReg& r : bounds_readers()) {
    if (e != cudaSuccess) break;
    BoundsRecord rec{};
    e = r.reader(&rec, reset);
    if (e == cudaSuccess && rec.count) {
      if (*count == 0) {
        *first = rec;
        *file = r.file;
      }
      *count += rec.count;
    }
  }
  return e;
}

int register_bounds_reader(BoundsReader reader, const char* file) {
  bounds_readers().push_back({reader, file});
  return (int)bounds_readers().size();
}

// TOPO_E_BOUNDS when an index check of the debug build has recorded a violation (what: the
// entry point), else st.
topo_status bounds_status(topo_status st, const char* what) {
#ifdef TOPO_BOUNDS_CHECK
  unsigned long long count = 0;
  BoundsRecord rec{};
  const char* file = "";
  cudaError_t e = read_bounds(&count, &rec, &file, false);
  if (e != cudaSuccess) return cuda_status(e, what);
  if (count) {
    set_error(std::string(what) + ": " + std::to_string(count) +
              " index(es) out of range, the first " + std::to_string(rec.index) + " of size " +
              std::to_string(rec.size) + " at " + file + ":" + std::to_string(rec.line));
    return TOPO_E_BOUNDS;
  }
#else
  (void)what;
#endif
  return st;
}

}  // namespace topo

using namespace topo;

namespace {

double w1h(int p, int q) {
  const int d = p - 2 * q;
  return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0);
}
int lox(int a) { return ((a & 3) == 1 || (a & 3) == 2) ? 1 : 0; }
int loy(int a) { return ((a & 3) >= 2) ? 1 : 0; }
int loz(int a) { return a >> 2; }

// C_c = P_c^T K0 P_c for the 2^dim children of a coarse element.
void child_matrices(int dim, const double* K0, std::vector<double>& C) {
  const int NN = dim == 2 ? 4 : 8, NE = NN * dim;
  C.assign((size_t)NN * NE * NE, 0.0);
  for (int c = 0; c < NN; ++c) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
    std::vector<double> W(NN * NN);
    for (int a = 0; a < NN; ++a)
      for (int A = 0; A < NN; ++A) {
        double w = w1h(cx + lox(a), lox(A)) * w1h(cy + loy(a), loy(A));
        if (dim == 3) w *= w1h(cz + loz(a), loz(A));
        W[a * NN + A] = w;
      }
    for (int I = 0; I < NE; ++I)
      for (int J = 0; J < NE; ++J) {
        const int A = I / dim, al = I % dim, B = J / dim, be = J % dim;
        double acc = 0.0;
        for (int a = 0; a < NN; ++a)
          for (int b = 0; b < NN; ++b)
            acc += W[a * NN + A] * K0[(a * dim + al) * NE + b * dim + be] * W[b * NN + B];
        C[(size_t)c * NE * NE + I * NE + J] = acc;
      }
  }
}

// C2_f = W_f^T K0 W_f for the 4^dim fine elements f two levels below a coarse element, with the
// composite node weights W_f[a][A] = sum_b W_c2[a][b] W_c1[b][A] (f = c1 * 2^dim + c2).
void grandchild_matrices(int dim, const double* K0, std::vector<double>& C2) {
  const int NN = dim == 2 ? 4 : 8, NE = NN * dim;
  auto weights = [&](int c, std::vector<double>& W) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
    W.assign(NN * NN, 0.0);
    for (int a = 0; a < NN; ++a)
      for (int A = 0; A < NN; ++A) {
        double w = w1h(cx + lox(a), lox(A)) * w1h(cy + loy(a), loy(A));
        if (dim == 3) w *= w1h(cz + loz(a), loz(A));
        W[a * NN + A] = w;
      }
  };
  C2.assign((size_t)NN * NN * NE * NE, 0.0);
  std::vector<double> W1, W2, Wf(NN * NN);
  for (int c1 = 0; c1 < NN; ++c1) {
    weights(c1, W1);
    for (int c2 = 0; c2 < NN; ++c2) {
      weights(c2, W2);
      for (int a = 0; a < NN; ++a)
        for (int A = 0; A < NN; ++A) {
          double w = 0.0;
          for (int b = 0; b < NN; ++b) w += W2[a * NN + b] * W1[b * NN + A];
          Wf[a * NN + A] = w;
        }
      double* Cf = C2.data() + (size_t)(c1 * NN + c2) * NE * NE;
      for (int I = 0; I < NE; ++I)
        for (int J = 0; J < NE; ++J) {
          const int A = I / dim, al = I % dim, B = J / dim, be = J % dim;
          double acc = 0.0;
          for (int a = 0; a < NN; ++a)
            for (int b = 0; b < NN; ++b)
              acc += Wf[a * NN + A] * K0[(a * dim + al) * NE + b * dim + be] * Wf[b * NN + B];
          Cf[I * NE + J] = acc;
        }
    }
  }
}

// Butterfly coefficients of the plane-stress Q1 K0 (see kernels_q1.cu) and a check that they
// reproduce the quadrature K0.
bool q1_coefficients(double E, double nu, const double* K0, Q1Coef& q) {
  const double c = E / (1.0 - nu * nu);
  const double D11 = c, D22 = c, D12 = c * nu, D33 = 0.5 * c * (1.0 - nu);
  q = Q1Coef{D11 / 4.0, D12 / 4.0, D22 / 4.0, D33 / 4.0, (D11 + D33) / 12.0, (D22 + D33) / 12.0,
             K0[0]};
  const double xi[4] = {-1, 1, 1, -1}, eta[4] = {-1, -1, 1, 1};
  double T[5][8] = {};
  for (int a = 0; a < 4; ++a) {
    T[0][2 * a] = xi[a];
    T[1][2 * a + 1] = eta[a];
    T[2][2 * a] = eta[a];
    T[2][2 * a + 1] = xi[a];
    T[3][2 * a] = xi[a] * eta[a];
    T[4][2 * a + 1] = xi[a] * eta[a];
  }
  double Kh[5][5] = {};
  Kh[0][0] = q.c11;
  Kh[0][1] = Kh[1][0] = q.c12;
  Kh[1][1] = q.c22;
  Kh[2][2] = q.c33;
  Kh[3][3] = q.cH;
  Kh[4][4] = q.cHp;
  double scale = 0.0, err = 0.0;
  for (int i = 0; i < 8; ++i) {
    if (std::fabs(K0[i * 8 + i] - K0[0]) > 1e-14 * std::fabs(K0[0])) return false;
    for (int j = 0; j < 8; ++j) {
      double acc = 0.0;
      for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) acc += T[a][i] * Kh[a][b] * T[b][j];
      err = std::max(err, std::fabs(acc - K0[i * 8 + j]));
      scale = std::max(scale, std::fabs(K0[i * 8 + j]));
    }
  }
  return err <= 1e-14 * scale;
}

// The butterfly coefficients of a caller's 8 x 8 K0: T has mutually orthogonal rows (squared norms
// 4, 4, 8, 4, 4), so Khat_ab = T_a K0 T_b^T / (|T_a|^2 |T_b|^2) is the only candidate; the path is
// taken when Khat has the butterfly's pattern (the normal block on (X, Y'), scalars on G, H, H'),
// T^T Khat T reproduces K0 and the diagonal of K0 is constant (the on-the-fly Jacobi diagonal).
bool q1_coefficients_from_K0(const double* K0, Q1Coef& q) {
  const double xi[4] = {-1, 1, 1, -1}, eta[4] = {-1, -1, 1, 1};
  double T[5][8] = {};
  for (int a = 0; a < 4; ++a) {
    T[0][2 * a] = xi[a];
    T[1][2 * a + 1] = eta[a];
    T[2][2 * a] = eta[a];
    T[2][2 * a + 1] = xi[a];
    T[3][2 * a] = xi[a] * eta[a];
    T[4][2 * a + 1] = xi[a] * eta[a];
  }
  const double nrm[5] = {4, 4, 8, 4, 4};
  double Kh[5][5] = {}, scale = 0.0;
  for (int i = 0; i < 64; ++i) scale = std::max(scale, std::fabs(K0[i]));
  if (!(scale > 0.0)) return false;
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) {
      double acc = 0.0;
      for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) acc += T[a][i] * K0[i * 8 + j] * T[b][j];
      Kh[a][b] = acc / (nrm[a] * nrm[b]);
    }
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) {
      const bool allowed = (a == b) || (a < 2 && b < 2);
      if (!allowed && std::fabs(Kh[a][b]) > 1e-14 * scale) return false;
    }
  double err = 0.0;
  for (int i = 0; i < 8; ++i) {
    if (std::fabs(K0[i * 8 + i] - K0[0]) > 1e-14 * scale) return false;
    for (int j = 0; j < 8; ++j) {
      double acc = 0.0;
      for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) {
          const bool allowed = (a == b) || (a < 2 && b < 2);
          if (allowed) acc += T[a][i] * Kh[a][b] * T[b][j];
        }
      err = std::max(err, std::fabs(acc - K0[i * 8 + j]));
    }
  }
  if (err > 1e-14 * scale) return false;
  q = Q1Coef{Kh[0][0], 0.5 * (Kh[0][1] + Kh[1][0]), Kh[1][1], Kh[2][2], Kh[3][3], Kh[4][4], K0[0]};
  return true;
}

// The element matrix of a descriptor: the caller's K0 or the analytic one.
void descriptor_K0(const topo_solver_desc* d, std::vector<double>& K0) {
  const int ne = d->dim == 2 ? 8 : 24;
  K0.assign((size_t)ne * ne, 0.0);
  if (d->K0)
    std::copy(d->K0, d->K0 + ne * ne, K0.begin());
  else
    element_stiffness_host(d->dim, d->E, d->nu, K0.data());
}

// Coarse mask by injection; check that every fixed fine DOF interpolates only from fixed coarse
// DOFs (then the element-local Galerkin product of the unmasked operators equals the masked one).
bool coarsen_mask(const Dims& df, const std::vector<uint8_t>& ff, std::vector<uint8_t>& fc,
                  std::string& why) {
  const int dim = df.dim;
  Dims dc{df.nx / 2, df.ny / 2, dim == 3 ? df.nz / 2 : 1, dim};
  fc.assign((size_t)dc.dofs(), 0);
  const int fnx = df.nx + 1, fny = df.ny + 1, cnx = dc.nx + 1, cny = dc.ny + 1;
  for (long long cn = 0; cn < dc.nodes(); ++cn) {
    const int I = (int)(cn % cnx), J = (int)((cn / cnx) % cny), K = (int)(cn / ((long long)cnx * cny));
    const long long fn = 2 * I + (long long)fnx * (2 * J + (long long)fny * 2 * K);
    for (int c = 0; c < dim; ++c) fc[dim * cn + c] = ff[dim * fn + c] ? 1 : 0;
  }
  for (long long fnode = 0; fnode < df.nodes(); ++fnode) {
    const int i = (int)(fnode % fnx), j = (int)((fnode / fnx) % fny), k = (int)(fnode / ((long long)fnx * fny));
    for (int c = 0; c < dim; ++c) {
      if (!ff[dim * fnode + c]) continue;
      const int kmax = dim == 3 ? ((k + 1) >> 1) : 0;
      for (int K = k >> 1; K <= kmax; ++K)
        for (int J = j >> 1; J <= ((j + 1) >> 1); ++J)
          for (int I = i >> 1; I <= ((i + 1) >> 1); ++I) {
            const long long cn = I + (long long)cnx * (J + (long long)cny * K);
            if (!fc[dim * cn + c]) {
              why = "fixed DOF mask is not compatible with geometric coarsening";
              return false;
            }
          }
    }
  }
  return true;
}

template <typename T>
struct Prec;
template <>
struct Prec<double> {
  static const double* K0(topo_solver* s) { return s->K0; }
  static const double* x(topo_solver* s) { return s->x; }
  static const double* Ae(const Level& l) { return l.Ae; }
  static const double* invd(const Level& l) { return l.invd; }
};
template <>
struct Prec<float> {
  static const float* K0(topo_solver* s) { return s->K0f; }
  static const float* x(topo_solver* s) { return s->x32; }
  static const float* Ae(const Level& l) { return l.Ae32; }
  static const float* invd(const Level& l) { return l.invd32; }
};

// Arrow vector w of a level and the fine-level rank-one data in the V-cycle precision.
template <typename TV>
const TV* arrow_w(const Level& l);
template <>
const double* arrow_w<double>(const Level& l) { return l.w; }
template <>
const float* arrow_w<float>(const Level& l) { return l.w32; }

template <typename TV>
struct ArrowFine;
template <>
struct ArrowFine<double> {
  static const double* g(topo_solver* s) { return s->g; }
  static const double* Dinv(topo_solver* s) { return s->Dinv; }
  static double* se(topo_solver* s) { return s->se; }
};
template <>
struct ArrowFine<float> {
  static const float* g(topo_solver* s) { return s->g32; }
  static const float* Dinv(topo_solver* s) { return s->Dinv32; }
  static float* se(topo_solver* s) { return s->se32; }
};

// External event-record node around a profiled kernel (kind, slot of the captured iteration); a
// plain record during capture would only track dependencies.
topo_status prof_mark(topo_solver* s, int kind, int end) {
  if (!s->profiling || s->prof_slot < 0 || !((s->prof_mask >> kind) & 1u)) return TOPO_OK;
  const size_t i = ((size_t)kind * s->graph_iters + s->prof_slot) * 2 + end;
  TOPO_CUDA(cudaEventRecordWithFlags(s->prof_ev[i], s->st, cudaEventRecordExternal));
  return TOPO_OK;
}

// The finest-level Q1 sweeps: two node columns per lane for FP32 vectors (kernels_q1w.cu, the
// same outputs), one column per lane otherwise (kernels_q1.cu).
template <typename TV>
cudaError_t q1_apply(const topo_solver* s, int nx, int ny, int mode, const TV* x, const TV* v,
                     const TV* b, TV* y, TV omega, const uint8_t* fixed, int nrhs,
                     const CgScalars* sc) {
  if constexpr (std::is_same<TV, float>::value) {
    if (s->q1_wide && s->fixed_pad)
      return launch_q1w_apply(nx, ny, mode, s->q1, x, v, b, y, omega, s->fixed_pad, nrhs, sc,
                              s->st, s->sweep_rows);
  }
  return launch_q1_apply<TV>(nx, ny, mode, s->q1, x, v, b, y, omega, fixed, nrhs, sc, s->st);
}
template <typename TV>
cudaError_t q1_fused(const topo_solver* s, int nx, int ny, int mode, const TV* x, const TV* t,
                     const TV* zc, const TV* b, TV* y, TV omega, const uint8_t* fixed, int nrhs,
                     const CgScalars* sc) {
  if constexpr (std::is_same<TV, float>::value) {
    if (s->q1_wide && s->fixed_pad)
      return launch_q1w_fused(nx, ny, mode, s->q1, x, t, zc, b, y, omega, s->fixed_pad, nrhs, sc,
                              s->st, s->sweep_rows);
  }
  return launch_q1_fused<TV>(nx, ny, mode, s->q1, x, t, zc, b, y, omega, fixed, nrhs, sc, s->st);
}
template <typename TV>
cudaError_t q1_resrestrict(const topo_solver* s, int nx, int ny, const TV* x, const TV* v,
                           const TV* b, TV* bc, const uint8_t* fixed, const uint8_t* fixed_c,
                           int nrhs, const CgScalars* sc) {
  if constexpr (std::is_same<TV, float>::value) {
    if (s->q1_wide && s->fixed_pad)
      return launch_q1w_resrestrict(nx, ny, s->q1, x, v, b, bc, s->fixed_pad, fixed_c, nrhs, sc,
                                    s->st, s->sweep_rows);
  }
  return launch_q1_resrestrict<TV>(nx, ny, s->q1, x, v, b, bc, fixed, fixed_c, nrhs, sc, s->st);
}
template <typename TV>
cudaError_t q1_smooth_beta(const topo_solver* s, int nx, int ny, const TV* x, const TV* v,
                           const TV* b, TV* y, TV omega, const uint8_t* fixed, int nrhs,
                           double* partials, unsigned* counters, CgScalars* sc) {
  // (the two-column form of this sweep, with its FP64 residual read for r~^T y~, measured slower
  // than the one-column kernel: 31.4 against 27.3 us per launch on 2048 x 1024; with the integer
  // conversions in both, the 2048 x 1024 step took 4.61 against 4.57 ms)
  return launch_q1_smooth_beta<TV>(nx, ny, s->q1, x, v, b, y, omega, fixed, nrhs, s->r, partials,
                                   counters, sc, s->st);
}

// Whether a level keeps an element-major copy of its V-cycle matrices for the single-block deep
// tail: 2D K systems, stored matrices, not the coarsest, at most kTailNodes nodes.
bool aem_level(int dim, bool arrow, bool coarsest, bool matrix_free, long long nodes) {
  return dim == 2 && !arrow && !coarsest && !matrix_free && nodes <= kTailNodes;
}

// TOPO_HEX_OUTER=tile: the 3D outer operator in the tile form (one launch, no force buffer, the
// same q).  The default is the two-kernel form with the force buffer: on 128 x 64 x 64 with 8
// right-hand sides the tile form took 848 us per launch against 349 + 200 us for the pair (it
// computes about 30% of the elements twice, and the pair-arithmetic element product is the cost).
bool hex_buffered_env() {
  const char* v = std::getenv("TOPO_HEX_OUTER");
  return !(v && std::string(v) == "tile");
}

// TOPO_HEX_SWEEP=node|dense|tc|wht: the 3D finest V-cycle operator (node-parallel; tile with the
// rows of K0, the same bits as node-parallel; the same product on the tensor cores, 3 x TF32;
// tile in the Walsh-Hadamard basis, when K0 has its
// structure: the default, 168 + 157 us against 238 + 201 us per V-cycle on 128 x 64 x 64 with 8
// right-hand sides; the dense tile form was the slowest).
int hex_sweep_env(bool hex_ok) {
  const char* v = std::getenv("TOPO_HEX_SWEEP");
  const std::string w = v ? v : "";
  if (w == "dense") return 1;
  if (w == "tc") return 3;  // the dense product on the tensor cores (FP32 V-cycle; FP64: dense)
  if (w == "node" || !hex_ok) return 0;
  return 2;
}

// Operator application on level k (mode as launch_apply): the warp-sweep Q1 kernels on the 2D
// finest level, the matrix-free first coarse level in mixed precision, the Z operator (element
// rank-one terms and lambda row) for IP systems, the generic element-matrix kernels elsewhere.
template <typename TV>
topo_status apply_level(topo_solver* s, int k, int mode, const TV* v, const TV* b, TV* y,
                        const CgScalars* sc, const TV* zc = nullptr, int nrhs = 0) {
  Level& lv = s->L[k];
  // nrhs: the vectors v, b, y hold this many right-hand sides (0: the solver's batch); the
  // build-time power iteration applies the operator to a single vector
  if (nrhs <= 0) nrhs = s->nrhs;
  // adaptive damping: omega_k is folded into invd at build time (and read from the device for the
  // lambda entry), so the kernels take omega = 1
  const TV omega = lv.omega_dev ? TV(1) : (TV)s->desc.omega;
  if (s->arrow) {
    if (k == 0) {
      TOPO_CUDA(launch_z_apply_fine<TV>(lv.d, mode, Prec<TV>::K0(s), Prec<TV>::x(s),
                                        ArrowFine<TV>::g(s), ArrowFine<TV>::Dinv(s),
                                        ArrowFine<TV>::se(s), v, b, y, Prec<TV>::invd(lv), omega,
                                        lv.fixed, s->zll, s->partials, s->counters, sc, s->st,
                                        lv.omega_dev));
      return TOPO_OK;
    }
    TOPO_CUDA(launch_apply_arrow<TV>(lv.d, mode, Prec<TV>::Ae(lv), v, b, y, Prec<TV>::invd(lv),
                                     omega, lv.fixed, arrow_w<TV>(lv), s->zll,
                                     (double)s->desc.omega, lv.omega_dev, s->partials,
                                     s->counters, sc, s->st));
    return TOPO_OK;
  }
  if (k == 0 && s->q1_ok) {
    TOPO_CUDA(q1_apply<TV>(s, lv.d.nx, lv.d.ny, mode, Prec<TV>::x(s), v, b, y, omega, lv.fixed,
                           nrhs, sc));
    return TOPO_OK;
  }
  if (k == 1 && s->l1_free && std::is_same<TV, float>::value) {
    if (s->q1_ok)
      TOPO_CUDA(launch_q1g_apply(lv.d.nx, lv.d.ny, mode, s->q1, s->x32, (const float*)v,
                                 (const float*)b, (float*)y, (float)omega, s->L[1].invd32,
                                 lv.fixed, nrhs, sc, s->st, (const float*)zc));
    else
      TOPO_CUDA(launch_apply_l1<float>(lv.d, mode, s->C32, s->x32, (const float*)v,
                                       (const float*)b, (float*)y, s->L[1].invd32, (float)omega,
                                       lv.fixed, nrhs, sc, s->st));
    return TOPO_OK;
  }
  if (k == 1 && s->l1_free) {  // FP64 products on the matrix-free level (build-time power iteration)
    TOPO_CUDA(launch_apply_l1<double>(lv.d, mode, s->C, s->x, (const double*)v, (const double*)b,
                                      (double*)y, lv.invd, (double)omega, lv.fixed, nrhs, sc,
                                      s->st));
    return TOPO_OK;
  }
  if (k == 0 && s->hex_sweep && mode <= 2) {  // 3D finest level: the tile form
    const int form = s->hex_sweep == 2 ? 0 : (s->hex_sweep == 3 && sizeof(TV) == 4 ? 2 : 1);
    TOPO_CUDA(launch_hex_tile_sweep<TV>(lv.d, mode, form, s->hex, Prec<TV>::K0(s),
                                        Prec<TV>::x(s), v, b, y, Prec<TV>::invd(lv), omega,
                                        lv.fixed, nrhs, sc, s->st));
    return TOPO_OK;
  }
  const TV* x = k == 0 ? Prec<TV>::x(s) : nullptr;
  const TV* Ae = k == 0 ? nullptr : Prec<TV>::Ae(lv);
  if (k >= 1 && !Ae) {
    set_error("apply_level: level " + std::to_string(k) + " holds no element matrices in this precision");
    return TOPO_E_INVALID_ARG;
  }
  TOPO_CUDA(launch_apply<TV>(lv.d, mode, Prec<TV>::K0(s), x, Ae, v, b, y, Prec<TV>::invd(lv), omega,
                             lv.fixed, nrhs, sc, s->st));
  return TOPO_OK;
}

// One V-cycle at level k with right-hand side b (Algorithm MG, function mgm, from z = 0).
// First level of the fused deep part of the V-cycle in precision TV, or -1: 2D K systems with
// Jacobi smoothing, element matrices in TV on every fused level above the coarsest, at most
// kTailNodes nodes on the first fused level and kTailMax fused levels.
template <typename TV>
int tail_level(const topo_solver* s) {
  if (!s->fuse_on || !s->tail_ok || s->dim != 2 || s->arrow || s->desc.smoother != 0) return -1;
  const int last = s->nlev - 1;
  for (int k = 1; k < last; ++k) {
    if (s->L[k].d.nodes() > kTailNodes || s->nlev - k > kTailMax) continue;
    bool ok = true;  // (the fused kernel takes one damping for all its levels)
    for (int j = k; j < last; ++j)
      ok = ok && Prec<TV>::Ae(s->L[j]) && Prec<TV>::invd(s->L[j]) && !s->L[j].omega_dev;
    if (ok) return k;
  }
  return -1;
}

// fuse_beta: the last smoothing sweep of the finest level also forms r~^T y~ and beta (the CG
// direction update then needs only the p kernel).
template <typename TV>
topo_status vcycle(topo_solver* s, int k, const TV* b, TV** result, const CgScalars* sc,
                   bool fuse_beta = false) {
  Level& lv = s->L[k];
  const int nrhs = s->nrhs;
  TV* zk = (TV*)lv.z;
  if (k == s->nlev - 1) {
    TOPO_CUDA(launch_dense_solve<TV>(s->nc + (s->arrow ? 1 : 0), s->Ainv, s->AinvDF, b, zk, nrhs,
                                     sc, s->st));
    *result = zk;
    return TOPO_OK;
  }
  TV* cur = zk;
  TV* oth = (TV*)lv.t;
  const int nu1 = s->desc.nu1, nu2 = s->desc.nu2;
  if (k == tail_level<TV>(s)) {  // this level and all below in one cluster launch
    TailArgs<TV> a = {};
    a.nl = s->nlev - k;
    a.nu1 = nu1;
    a.nu2 = nu2;
    a.nc = s->nc;
    a.omega = (TV)s->desc.omega;
    a.Ainv = s->Ainv;
    a.AinvDF = s->AinvDF;
    a.wait_ns = s->wait_ns;
    for (int j = 0; j < a.nl; ++j) {
      Level& l = s->L[k + j];
      a.d[j] = l.d;
      a.Ae[j] = Prec<TV>::Ae(l);
      a.Aem[j] = (const TV*)l.Aem;
      a.invd[j] = Prec<TV>::invd(l);
      a.fixed[j] = l.fixed;
      a.b[j] = j == 0 ? const_cast<TV*>(b) : (TV*)l.b;
      a.z[j] = (TV*)l.z;
      a.t[j] = (TV*)l.t;
    }
    if (tail1_layout<TV>(a)) {  // all fused levels in one block's shared memory
      TOPO_CUDA(launch_vcycle_tail1<TV>(a, nrhs, sc, s->st));
      *result = zk;
      return TOPO_OK;
    }
    TOPO_CUDA(launch_vcycle_tail<TV>(a, nrhs, sc, s->st));
    // the iterate ends where the unfused cycle leaves it: one swap per plain sweep
    const int swaps = (nu1 >= 1 ? nu1 - 1 : 0) + nu2;
    *result = (swaps % 2 == 0) ? cur : oth;
    return TOPO_OK;
  }
  if (lv.lam_dev) {  // Chebyshev smoothing, the same polynomial before and after the correction
    const long long nv = lv.n;
    const TV* inv = Prec<TV>::invd(lv);
    for (int it = 0; it < nu1; ++it) {
      const TV* t = b;
      if (it > 0) {
        TOPO_TRY(apply_level<TV>(s, k, 1, cur, b, oth, sc));
        t = oth;
      }
      TOPO_CUDA(launch_cheb_update<TV>(nv, nrhs, it, it == 0 ? 1 : 0, lv.lam_dev, 4.0, inv, t,
                                       (TV*)lv.cd, cur, lv.fixed, sc, s->st));
    }
    if (nu1 == 0) TOPO_CUDA(cudaMemsetAsync(cur, 0, sizeof(TV) * s->vlen(k) * nrhs, s->st));
    TOPO_TRY(apply_level<TV>(s, k, 1, cur, b, oth, sc));
    Level& lc = s->L[k + 1];
    TOPO_CUDA(launch_restrict<TV>(lv.d, oth, (TV*)lc.b, lc.fixed, nrhs, sc, s->st, s->arrow));
    TV* zc = nullptr;
    TOPO_TRY(vcycle<TV>(s, k + 1, (const TV*)lc.b, &zc, sc, false));
    TOPO_CUDA(launch_prolong_add<TV>(lv.d, zc, cur, lv.fixed, nrhs, sc, s->st, s->arrow));
    for (int it = 0; it < nu2; ++it) {
      TOPO_TRY(apply_level<TV>(s, k, 1, cur, b, oth, sc));
      TOPO_CUDA(launch_cheb_update<TV>(nv, nrhs, it, 0, lv.lam_dev, 4.0, inv, oth, (TV*)lv.cd,
                                       cur, lv.fixed, sc, s->st));
    }
    *result = cur;
    return TOPO_OK;
  }
  const bool fine = (k == 0);
  // finest 2D Q1 level: the first two sweeps, and the prolongation with the first post-sweep, as
  // single fused kernels (the same bits)
  const bool fine_fused = fine && s->fuse_on && s->q1_ok && !s->arrow;
  // the matrix-free first coarse level (2D mixed): both fusions in its warp sweep
  const bool l1_fused = k == 1 && s->fuse_on && s->l1_free && s->q1_ok && !s->arrow &&
                        std::is_same<TV, float>::value;
  // coarse 2D levels with stored element matrices: the first two sweeps as one kernel (mode 4),
  // and the prolongation with the first post-sweep (v = z + P z_c formed once per neighbour node
  // from a 3 x 3 coarse patch, k_apply2_prolong).
  // IP systems: the first two sweeps, with the lambda row in the kernel (k_apply_arrow).
  const bool coarse_fused = !fine && s->fuse_on && s->dim == 2 && !(k == 1 && s->l1_free) &&
                            Prec<TV>::Ae(lv) != nullptr;
  bool sweep_timed = false;  // profiling: the first smoothing kernel of the finest level
  if (nu1 >= 2 && fine_fused) {
    TOPO_TRY(prof_mark(s, 1, 0));
    TOPO_CUDA(q1_fused<TV>(s, lv.d.nx, lv.d.ny, 4, Prec<TV>::x(s), nullptr, nullptr, b, oth,
                           (TV)s->desc.omega, lv.fixed, nrhs, sc));
    TOPO_TRY(prof_mark(s, 1, 1));
    sweep_timed = true;
    std::swap(cur, oth);
    for (int it = 2; it < nu1; ++it) {
      TOPO_TRY(apply_level<TV>(s, k, 2, cur, b, oth, sc));
      std::swap(cur, oth);
    }
  } else if (nu1 >= 2 && (coarse_fused || l1_fused)) {
    TOPO_TRY(apply_level<TV>(s, k, 4, cur, b, oth, sc));
    std::swap(cur, oth);
    for (int it = 2; it < nu1; ++it) {
      TOPO_TRY(apply_level<TV>(s, k, 2, cur, b, oth, sc));
      std::swap(cur, oth);
    }
  } else if (nu1 >= 1) {
    TOPO_TRY(apply_level<TV>(s, k, 3, cur, b, cur, sc));
    for (int it = 1; it < nu1; ++it) {
      const bool t = fine && !sweep_timed;
      if (t) TOPO_TRY(prof_mark(s, 1, 0));
      TOPO_TRY(apply_level<TV>(s, k, 2, cur, b, oth, sc));
      if (t) TOPO_TRY(prof_mark(s, 1, 1));
      sweep_timed = sweep_timed || t;
      std::swap(cur, oth);
    }
  } else {
    TOPO_CUDA(cudaMemsetAsync(cur, 0, sizeof(TV) * s->vlen(k) * nrhs, s->st));
  }
  Level& lc = s->L[k + 1];
  if (fine_fused) {  // residual and restriction in one pass (the residual is not stored)
    TOPO_TRY(prof_mark(s, 2, 0));
    TOPO_CUDA(q1_resrestrict<TV>(s, lv.d.nx, lv.d.ny, Prec<TV>::x(s), cur, b, (TV*)lc.b,
                                 lv.fixed, lc.fixed, nrhs, sc));
    TOPO_TRY(prof_mark(s, 2, 1));
  } else {
    if (fine) TOPO_TRY(prof_mark(s, 2, 0));
    TOPO_TRY(apply_level<TV>(s, k, 1, cur, b, oth, sc));
    if (fine) TOPO_TRY(prof_mark(s, 2, 1));
    if (fine) TOPO_TRY(prof_mark(s, 3, 0));
    TOPO_CUDA(launch_restrict<TV>(lv.d, oth, (TV*)lc.b, lc.fixed, nrhs, sc, s->st, s->arrow));
    if (fine) TOPO_TRY(prof_mark(s, 3, 1));
  }
  TV* zc = nullptr;
  const int sub_kind = k <= 5 ? 6 + k : -1;  // levels >= k + 1
  if (sub_kind > 0) TOPO_TRY(prof_mark(s, sub_kind, 0));
  TOPO_TRY(vcycle<TV>(s, k + 1, (const TV*)lc.b, &zc, sc, false));
  if (sub_kind > 0) TOPO_TRY(prof_mark(s, sub_kind, 1));
  int it0 = 0;
  if (fine_fused && nu2 >= 1 && !(fuse_beta && nu2 == 1)) {
    TOPO_TRY(prof_mark(s, 4, 0));
    TOPO_CUDA(q1_fused<TV>(s, lv.d.nx, lv.d.ny, 5, Prec<TV>::x(s), cur, zc, b, oth,
                           (TV)s->desc.omega, lv.fixed, nrhs, sc));
    TOPO_TRY(prof_mark(s, 4, 1));
    std::swap(cur, oth);
    it0 = 1;
  } else if (l1_fused && nu2 >= 1) {
    TOPO_TRY(apply_level<TV>(s, k, 5, cur, b, oth, sc, zc));
    std::swap(cur, oth);
    it0 = 1;
  } else if (coarse_fused && !s->arrow && nu2 >= 1 && s->coarse_prolong &&
             lv.d.nodes() <= kApply2ProlongNodes) {
    const TV omega = lv.omega_dev ? TV(1) : (TV)s->desc.omega;
    TOPO_CUDA(launch_apply2_prolong<TV>(lv.d, Prec<TV>::Ae(lv), cur, zc, b, oth,
                                        Prec<TV>::invd(lv), omega, lv.fixed, nrhs, sc, s->st));
    std::swap(cur, oth);
    it0 = 1;
  } else {
    if (fine) TOPO_TRY(prof_mark(s, 4, 0));
    TOPO_CUDA(launch_prolong_add<TV>(lv.d, zc, cur, lv.fixed, nrhs, sc, s->st, s->arrow));
    if (fine) TOPO_TRY(prof_mark(s, 4, 1));
  }
  for (int it = it0; it < nu2; ++it) {
    if (fuse_beta && k == 0 && it == nu2 - 1 && s->q1_ok) {
      TOPO_CUDA(q1_smooth_beta<TV>(s, lv.d.nx, lv.d.ny, Prec<TV>::x(s), cur, b, oth,
                                   (TV)s->desc.omega, lv.fixed, nrhs, s->partials, s->counters,
                                   const_cast<CgScalars*>(sc)));
    } else if (fuse_beta && k == 0 && it == nu2 - 1) {  // the 3D tile sweep with r~^T y~, beta
      const TV omega = lv.omega_dev ? TV(1) : (TV)s->desc.omega;
      TOPO_CUDA(launch_hex_tile_sweep_beta<TV>(lv.d, s->hex_sweep == 2 ? 0 : 1, s->hex,
                                               Prec<TV>::K0(s), Prec<TV>::x(s), cur, b, oth,
                                               Prec<TV>::invd(lv), omega, lv.fixed, nrhs,
                                               const_cast<CgScalars*>(sc), s->r, s->partials,
                                               s->counters, s->st));
    } else {
      const bool t = fine && !sweep_timed;
      if (t) TOPO_TRY(prof_mark(s, 1, 0));
      TOPO_TRY(apply_level<TV>(s, k, 2, cur, b, oth, sc));
      if (t) TOPO_TRY(prof_mark(s, 1, 1));
      sweep_timed = sweep_timed || t;
    }
    std::swap(cur, oth);
  }
  *result = cur;
  return TOPO_OK;
}

// Preconditioner on the PCG residual r: y = M^{-1} r (result pointer returned).
template <typename TV>
topo_status precondition(topo_solver* s, const CgScalars* sc, void** y, bool fuse_beta = false) {
  TV* out = nullptr;
  const TV* b = std::is_same<TV, double>::value ? (const TV*)s->r : (const TV*)s->rv;
  TOPO_TRY(vcycle<TV>(s, 0, b, &out, sc, fuse_beta));
  *y = out;
  return TOPO_OK;
}

// The outer CG's operator y = A v: the level-0 operator, or for the SIMP model (Sec. 9) the exact Z
// with the filter, whose element-local approximation the hierarchy holds.
topo_status apply_outer(topo_solver* s, const double* v, double* y, const CgScalars* sc) {
  if (s->simp.on) {
    const Level& l0 = s->L[0];
    TOPO_CUDA(launch_simp_z_apply(l0.d, s->K0, s->x, s->g, s->simp.Dinv, s->simp.invS,
                                  s->simp.rmin, s->simp.R, s->simp.ea, s->simp.eb, s->se, v, y,
                                  l0.fixed, s->partials, s->counters, sc, s->st,
                                  s->outer_df != 0));
    return TOPO_OK;
  }
  if (s->arrow && s->outer_df) {
    const Level& l0 = s->L[0];
    TOPO_CUDA(launch_z_apply_fine_df(l0.d, s->K0, s->x, s->g, s->Dinv, s->se, v, y, l0.fixed,
                                     s->zll, s->partials, s->counters, sc, s->st));
    return TOPO_OK;
  }
  return apply_level<double>(s, 0, 0, v, nullptr, y, sc);
}

// One PCG iteration (q = A p, update, precondition, new direction), enqueued on s->st.
template <typename TV>
topo_status cg_iteration(topo_solver* s, int slot, double tol, int max_iter) {
  Level& l0 = s->L[0];
  const long long n = s->ncg();
  s->prof_slot = s->profiling ? slot : -1;
  TOPO_TRY(prof_mark(s, 0, 0));
  if (s->arrow) {
    TOPO_TRY(apply_outer(s, s->p, s->q, s->sc));
    TOPO_CUDA(launch_cg_alpha(n, 1, s->p, s->q, s->partials, s->counters, s->sc, s->st));
  } else if (s->q1_ok && s->outer_df && s->xdf) {
    TOPO_CUDA(launch_q1_apply_dot_df(l0.d.nx, l0.d.ny, s->q1, s->xdf, s->p, s->q, l0.fixed,
                                     s->nrhs, s->partials, s->counters, s->sc, s->st));
  } else if (s->q1_ok) {
    TOPO_CUDA(launch_q1_apply_dot(l0.d.nx, l0.d.ny, s->q1, s->x, s->p, s->q, l0.fixed, s->nrhs,
                                  s->partials, s->counters, s->sc, s->st));
  } else if (s->hex_ok && !s->hex_buffered) {
    const bool pairs = s->outer_df && s->xdf;
    TOPO_CUDA(launch_hex_tile_apply_dot(l0.d, s->hex, pairs ? (const void*)s->xdf : (const void*)s->x,
                                        pairs, s->p, s->q, l0.fixed, s->nrhs, s->partials,
                                        s->counters, s->sc, s->st));
  } else if (s->hex_ok && s->outer_df && s->xdf) {
    TOPO_CUDA(launch_hex_apply_dot_df(l0.d, s->hex, s->xdf, s->p, s->q, l0.fixed, s->nrhs,
                                      s->hexR, s->partials, s->counters, s->sc, s->st));
  } else if (s->hex_ok) {
    TOPO_CUDA(launch_hex_apply_dot(l0.d, s->hex, s->x, s->p, s->q, l0.fixed, s->nrhs, s->hexR,
                                   s->partials, s->counters, s->sc, s->st));
  } else {
    TOPO_CUDA(launch_apply_dot_fine(l0.d, s->K0, s->x, s->p, s->q, l0.fixed, s->nrhs, s->partials,
                                    s->counters, s->sc, s->st));
  }
  TOPO_TRY(prof_mark(s, 0, 1));
  TV* rv = std::is_same<TV, double>::value ? nullptr : (TV*)s->rv;
  TOPO_CUDA(launch_cg_update<TV>(n, s->nrhs, s->z, s->r, s->p, s->q, rv, s->partials, s->counters,
                                 s->sc, tol, max_iter, s->st));
  void* y = nullptr;
  // (2D: the Q1 sweeps; 3D: the tile sweeps of forms 1 and 2)
  const bool fuse_ok = s->q1_ok || (s->dim == 3 && (s->hex_sweep == 1 || s->hex_sweep == 2));
  const bool fuse = fuse_ok && !s->arrow && s->desc.nu2 >= 1 && !s->desc.flexible &&
                    s->nlev >= 2 && s->desc.smoother == 0;
  TOPO_TRY(prof_mark(s, 5, 0));
  TOPO_TRY(precondition<TV>(s, s->sc, &y, fuse));
  TOPO_TRY(prof_mark(s, 5, 1));
  s->yv = y;
  // (the direction kernel also applies this iteration's z += alpha p)
  if (fuse)
    TOPO_CUDA(launch_cg_p<TV>(n, s->nrhs, (const TV*)y, s->p, (TV*)s->yold, 0, s->sc, s->st,
                              s->z));
  else
    TOPO_CUDA(launch_cg_direction<TV>(n, s->nrhs, s->r, (const TV*)y, s->p, (TV*)s->yold,
                                      s->desc.flexible, s->partials, s->counters, s->sc, s->st,
                                      s->z));
  s->prof_slot = -1;
  return TOPO_OK;
}

// Capture whatever `body` enqueues on s->st into an executable graph; count its kernel nodes.
template <typename F>
topo_status capture(topo_solver* s, cudaGraphExec_t* exec, int* kernels, F body) {
  if (*exec) {
    cudaGraphExecDestroy(*exec);
    *exec = nullptr;
  }
  cudaGraph_t g = nullptr;
  TOPO_CUDA(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
  topo_status st = body();
  cudaError_t e = cudaStreamEndCapture(s->st, &g);
  if (st != TOPO_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
  int kn = 0;
  for (size_t i = 0; i < nn; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
  }
  *kernels = kn;
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate");
  return TOPO_OK;
}

// One graph per solve after the setup: a conditional while node whose body is one CG iteration
// followed by the loop-condition kernel.
template <typename TV>
topo_status capture_loop(topo_solver* s, double tol, int max_iter) {
  if (s->loop) {
    cudaGraphExecDestroy(s->loop);
    s->loop = nullptr;
  }
  cudaGraph_t g = nullptr;
  TOPO_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle handle;
  cudaError_t e = cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_status(e, "cudaGraphConditionalHandleCreate");
  }
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = handle;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &prm);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_status(e, "cudaGraphAddNode(conditional)");
  }
  cudaGraph_t body = prm.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(s->st, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_status(e, "cudaStreamBeginCaptureToGraph");
  }
  const bool prof = s->profiling;
  s->profiling = false;  // no event nodes inside a conditional body
  topo_status st = cg_iteration<TV>(s, 0, tol, max_iter);
  s->profiling = prof;
  if (st == TOPO_OK) {
    cudaError_t le = launch_loop_cond(handle, s->sc, s->nrhs, max_iter, s->st);
    if (le != cudaSuccess) st = cuda_status(le, "launch_loop_cond");
  }
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(s->st, &captured);
  if (st != TOPO_OK) {
    cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_status(e, "cudaStreamEndCapture(loop body)");
  }
  size_t nn = 0;
  cudaGraphGetNodes(body, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) cudaGraphGetNodes(body, nodes.data(), &nn);
  int kn = 0;
  for (size_t i = 0; i < nn; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
  }
  s->loop_kernels = kn;
  e = cudaGraphInstantiate(&s->loop, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate(loop)");
  return TOPO_OK;
}

topo_status launch_graph(topo_solver* s, cudaGraphExec_t g, int kernels) {
  TOPO_CUDA(cudaGraphLaunch(g, s->st));
  s->launches += (unsigned long long)kernels;
  return TOPO_OK;
}

template <typename TV>
topo_status cg_setup(topo_solver* s, int use_x0, double tol, int max_iter) {
  const long long n = s->ncg();
  const int nrhs = s->nrhs;
  if (use_x0) {  // (from z = 0 the start vectors come from launch_cg_init_zero before the graph)
    TOPO_TRY(apply_outer(s, s->z, s->q, nullptr));
    TOPO_CUDA(launch_cg_init(n, nrhs, s->bbuf, s->z, s->r, s->q, use_x0, s->partials,
                             s->counters, s->sc, tol, max_iter, s->st));
    if (!std::is_same<TV, double>::value)
      TOPO_CUDA(launch_convert_d2f(s->r, (float*)s->rv, n * nrhs, s->st));
  }
  void* y = nullptr;
  TOPO_TRY(precondition<TV>(s, s->sc, &y));
  TOPO_CUDA(launch_cg_start_p<TV>(n, nrhs, s->r, (const TV*)y, s->p, (TV*)s->yold,
                                  s->desc.flexible, s->partials, s->counters, s->sc, s->st));
  return TOPO_OK;
}

template <typename TV>
topo_status solve_impl(topo_solver* s, const double* b, double* u, double tol, int use_x0,
                       topo_solve_info* info) {
  NvtxRange nvtx("topo: MGCG solve (Algorithm PCG)");
  const long long n = s->ncg();
  const int nrhs = s->nrhs;
  const int max_iter = s->desc.max_iter;
  const int ux = use_x0 ? 1 : 0;
  // The graphs bake in tol and max_iter: recapture when the tolerance changes.
  if (!s->setup[ux] || s->setup_tol[ux] != tol) {
    TOPO_TRY(capture(s, &s->setup[ux], &s->setup_kernels[ux],
                     [&]() { return cg_setup<TV>(s, ux, tol, max_iter); }));
    s->setup_tol[ux] = tol;
  }
  // Programmatic-launch attributes stay out of conditional bodies.
  const bool use_loop = s->graph_mode == 1 && !s->profiling && !s->no_loop && !pdl_enabled();
  if (use_loop && (!s->loop || s->loop_tol != tol)) {
    topo_status ls = capture_loop<TV>(s, tol, max_iter);
    if (ls != TOPO_OK) {  // conditional graphs unavailable: fall back to blocks of iterations
      cudaGetLastError();
      s->no_loop = true;
    } else {
      s->loop_tol = tol;
    }
  }
  if ((!use_loop || s->no_loop) && (!s->graph || s->graph_tol != tol)) {
    TOPO_TRY(capture(s, &s->graph, &s->graph_kernels, [&]() {
      for (int it = 0; it < s->graph_iters; ++it) TOPO_TRY(cg_iteration<TV>(s, it, tol, max_iter));
      return TOPO_OK;
    }));
    s->graph_tol = tol;
  }
  TOPO_CUDA(cudaEventRecord(s->ev_t0, s->st));
  // entries on fixed DOFs are ignored: the eliminated system has no equations there
  if (use_x0) {
    TOPO_CUDA(launch_mask_copy(n, s->L[0].n, nrhs, b, s->bbuf, s->L[0].fixed, s->st));
    TOPO_CUDA(launch_mask_copy(n, s->L[0].n, nrhs, u, s->z, s->L[0].fixed, s->st));
    s->launches += 2;
  } else {
    TOPO_CUDA(launch_cg_init_zero<TV>(n, s->L[0].n, nrhs, b, s->L[0].fixed, s->z, s->r,
                                      std::is_same<TV, double>::value ? nullptr : (TV*)s->rv,
                                      s->partials, s->counters, s->sc, tol, max_iter, s->st));
    s->launches += 1;
  }
  TOPO_TRY(launch_graph(s, s->setup[ux], s->setup_kernels[ux]));
  if (use_loop && !s->no_loop) {
    TOPO_CUDA(cudaGraphLaunch(s->loop, s->st));
    TOPO_CUDA(cudaMemcpyAsync(s->sc_host, s->sc, sizeof(CgScalars) * nrhs, cudaMemcpyDeviceToHost,
                              s->st));
    TOPO_CUDA(cudaStreamSynchronize(s->st));
    int executed = 0;
    for (int k = 0; k < nrhs; ++k) executed = std::max(executed, s->sc_host[k].iter);
    s->launches += (unsigned long long)s->loop_kernels * std::max(executed, 1);
  }
  int blocks = 0;
  const int max_blocks = (max_iter + s->graph_iters - 1) / s->graph_iters + 1;
  bool all_done = use_loop && !s->no_loop;
  int iter_before = 0;
  while (!all_done && blocks < max_blocks) {
    TOPO_TRY(launch_graph(s, s->graph, s->graph_kernels));
    ++blocks;
    TOPO_CUDA(cudaMemcpyAsync(s->sc_host, s->sc, sizeof(CgScalars) * nrhs, cudaMemcpyDeviceToHost,
                              s->st));
    TOPO_CUDA(cudaStreamSynchronize(s->st));
    all_done = true;
    int iter_after = 0;
    for (int k = 0; k < nrhs; ++k) {
      all_done = all_done && s->sc_host[k].done;
      iter_after = std::max(iter_after, s->sc_host[k].iter);
    }
    if (s->profiling) {
      const int ran = std::min(iter_after - iter_before, s->graph_iters);
      for (int kind = 0; kind < topo_solver::kProfKinds; ++kind)
        for (int slot = 0; slot < ran; ++slot) {
          const size_t i = ((size_t)kind * s->graph_iters + slot) * 2;
          float ms = 0.f;
          if (cudaEventElapsedTime(&ms, s->prof_ev[i], s->prof_ev[i + 1]) == cudaSuccess) {
            s->prof_ms[kind] += ms;
            s->prof_count[kind] += 1;
          } else {
            cudaGetLastError();  // kind not in this graph or timing unavailable: no sticky error
          }
        }
    }
    iter_before = iter_after;
  }
  // the iterate update of the last iteration (its direction kernel did not run)
  TOPO_CUDA(launch_cg_finish_z(n, nrhs, s->p, s->z, s->sc, s->st));
  s->launches += 1;
  if (u != s->z)
    TOPO_CUDA(cudaMemcpyAsync(u, s->z, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, s->st));
  TOPO_CUDA(cudaEventRecord(s->ev_t1, s->st));
  TOPO_CUDA(cudaEventSynchronize(s->ev_t1));
  topo_status worst = TOPO_OK;
  int it_max = 0;
  double rel_max = 0.0;
  for (int k = 0; k < nrhs; ++k) {
    const CgScalars& S = s->sc_host[k];
    if (S.iter > it_max) it_max = S.iter;
    if (S.rel > rel_max) rel_max = S.rel;
    if (S.status != TOPO_OK && worst == TOPO_OK) worst = (topo_status)S.status;
  }
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s->ev_t0, s->ev_t1);
    info->iterations = it_max;
    info->rel_residual = rel_max;
    info->wall_ms = ms;
    info->status = worst;
  }
  if (worst == TOPO_E_NOT_CONVERGED) set_error("CG reached max_iter before the tolerance");
  if (worst == TOPO_E_BREAKDOWN) set_error("CG breakdown (p^T A p <= 0 or a non-finite scalar)");
  if (worst == TOPO_E_TIMEOUT) set_error("a bounded device-side wait expired (V-cycle data copy)");
  return worst;
}

// Power iterations for lambda_max(D^{-1} A_k): from the fixed start vector on the first build, and
// from the previous build's vector afterwards (the matrices of consecutive IP Newton steps or OC
// iterations are close, so a few steps refine the estimate).
constexpr int kPowerCold = 15;
constexpr int kPowerWarm = 5;

topo_status enqueue_build(topo_solver* s, bool warm = false) {
  const int nl = s->nlev;
  const bool mixed = s->prec == TOPO_MIXED;
  cudaStream_t st = s->st;
  const long long m = s->L[0].m;
  const int ne2 = s->ne * s->ne;
  TOPO_CUDA(cudaMemsetAsync(s->info, 0, 4 * sizeof(int), st));
  TOPO_CUDA(launch_prepare_x(s->x, m, s->info + 1, mixed ? s->x32 : nullptr, s->xdf, st));
  if (s->arrow && mixed) {
    TOPO_CUDA(launch_convert_d2f(s->g, s->g32, m * s->ne, st));
    TOPO_CUDA(launch_convert_d2f(s->Dinv, s->Dinv32, m, st));
  }
  for (int k = 1; k < nl; ++k) {
    Level& lk = s->L[k];
    // FP32 hierarchy: FP32 products into Ae32 below the coarsest level, FP64 into Ae on it
    const bool f32 = s->h32 && !lk.Ae;
    if (k == 1) {
      if (f32 && lk.Ae32)
        TOPO_CUDA(launch_rap_from_fine<float>(s->L[0].d, s->C32, s->x32, lk.Ae32, st, nullptr,
                                              nullptr, s->C_host.data()));
      else if (lk.Ae)  // stored unless the first coarse level is applied matrix-free
        TOPO_CUDA(launch_rap_from_fine<double>(s->L[0].d, s->C, s->x, lk.Ae, st,
                                               s->arrow ? s->g : nullptr,
                                               s->arrow ? s->Dinv : nullptr, s->C_host.data()));
    } else if (k == 2 && s->C2) {
      if (f32)
        TOPO_CUDA(launch_rap2_from_fine<float>(s->L[0].d, s->C2f, s->x32, lk.Ae32, st,
                                               s->C2_host.data()));
      else
        TOPO_CUDA(launch_rap2_from_fine<double>(s->L[0].d, s->C2, s->x, lk.Ae, st,
                                                s->C2_host.data()));
    } else if (s->h32) {
      if (f32)
        TOPO_CUDA((launch_rap_coarse<float, float>(s->L[k - 1].d, s->L[k - 1].Ae32, lk.Ae32, st)));
      else
        TOPO_CUDA((launch_rap_coarse<float, double>(s->L[k - 1].d, s->L[k - 1].Ae32, lk.Ae, st)));
    } else {
      TOPO_CUDA((launch_rap_coarse<double, double>(s->L[k - 1].d, s->L[k - 1].Ae, lk.Ae, st)));
    }
    if (s->arrow)
      TOPO_CUDA(launch_restrict<double>(s->L[k - 1].d, s->L[k - 1].w, s->L[k].w, s->L[k].fixed, 1,
                                        nullptr, st, 0));
  }
  for (int k = 0; k < nl - 1; ++k) {
    Level& lv = s->L[k];
    // the 2D Q1 sweeps form the finest diagonal from x on the fly; only the power iteration and
    // the Chebyshev smoother read it from invd
    if (k == 0 && s->q1_ok && !s->arrow && !lv.omega_dev && !lv.lam_dev) continue;
    if (k >= 1 && !lv.Ae && lv.Ae32) {  // FP32 hierarchy level: FP32 diagonal only
      TOPO_CUDA(launch_inv_diag32(lv.d, lv.Ae32, lv.fixed, lv.invd32, st));
      continue;
    }
    if (k == 1 && !lv.Ae && mixed && !lv.omega_dev && !lv.lam_dev) {
      // the matrix-free first coarse level of an FP32 V-cycle: only its FP32 diagonal is read
      TOPO_CUDA(launch_inv_diag_l1<float>(lv.d, s->C32, s->x32, lv.fixed, lv.invd32, st));
      continue;
    }
    if (k == 1 && !lv.Ae)
      TOPO_CUDA(launch_inv_diag_l1<double>(lv.d, s->C, s->x, lv.fixed, lv.invd, st));
    else if (!(s->arrow && k == 0))  // the IP driver writes the finest diagonal of Z
      TOPO_CUDA(launch_inv_diag(lv.d, s->K0, k == 0 ? s->x : nullptr, lv.Ae, lv.fixed, lv.invd, st));
    if (lv.omega_dev || lv.lam_dev) {  // lambda_max(D^{-1} A_k) by power iteration
      const int ar = s->arrow ? 1 : 0;
      double* pv = s->pw_vec + s->pw_off[k];
      if (!warm) TOPO_CUDA(launch_power_init(lv.n, ar, pv, lv.fixed, st));
      const int steps = warm ? kPowerWarm : kPowerCold;
      for (int it = 0; it < steps; ++it) {
        TOPO_TRY(apply_level<double>(s, k, 0, pv, nullptr, s->q, nullptr, nullptr, 1));
        TOPO_CUDA(launch_power_step(lv.n, ar, pv, s->q, lv.invd, s->zll, s->r, s->partials,
                                    s->counters, s->pw_est, st));
      }
      if (lv.lam_dev)
        TOPO_CUDA(launch_power_store(s->pw_est, lv.lam_dev, st));
      else
        TOPO_CUDA(launch_power_finish(lv.n, s->pw_est, s->desc.omega, 4.0 / 3.0, lv.omega_dev,
                                      lv.invd, st));
    }
    if (mixed) {
      TOPO_CUDA(launch_convert_d2f(lv.invd, lv.invd32, lv.n, st));
      if (k >= 1 && lv.Ae32) TOPO_CUDA(launch_convert_d2f(lv.Ae, lv.Ae32, lv.m * ne2, st));
    }
  }
  if (s->arrow && mixed)
    for (int k = 0; k < nl; ++k) TOPO_CUDA(launch_convert_d2f(s->L[k].w, s->L[k].w32, s->L[k].n, st));
  for (int k = 1; k < nl - 1; ++k) {  // element-major copies for the single-block deep tail
    Level& lv = s->L[k];
    if (!lv.Aem) continue;
    if (mixed && lv.Ae32)
      TOPO_CUDA(launch_pack_element_major<float>(lv.m, lv.Ae32, (float*)lv.Aem, st));
    else if (!mixed && lv.Ae)
      TOPO_CUDA(launch_pack_element_major<double>(lv.m, lv.Ae, (double*)lv.Aem, st));
  }
  Level& lc = s->L[nl - 1];
  const bool fine_coarsest = (nl == 1);
  TOPO_CUDA(launch_assemble_dense(lc.d, s->K0, fine_coarsest ? s->x : nullptr, lc.Ae, lc.fixed,
                                  s->Adense, st, 0, s->arrow ? lc.w : nullptr, s->zll,
                                  (s->arrow && fine_coarsest) ? s->g : nullptr,
                                  (s->arrow && fine_coarsest) ? s->Dinv : nullptr));
  // K systems: Newton-Schulz inverse for small coarsest levels; IP systems keep the modified
  // Cholesky, whose pivot floor guards the nearly singular Schur complement of the multiplier.
  TOPO_CUDA(launch_cholesky_inverse(s->nc + (s->arrow ? 1 : 0), s->Adense, s->Ainv, s->info, st,
                                    s->Ascratch, s->info + 2, !s->arrow && s->Ascratch != nullptr));
  if (s->AinvDF) {  // the FP32 V-cycle's coarsest solve reads the inverse as float pairs
    const long long na = s->nc + (s->arrow ? 1 : 0);
    TOPO_CUDA(launch_split_df(s->Ainv, s->AinvDF, na * na, st));
  }
  return TOPO_OK;
}

topo_status build_hierarchy(topo_solver* s) {
  NvtxRange nvtx("topo: hierarchy build (Galerkin, Sec. 5.1)");
  const bool warm = s->pw_vec && s->pw_ready;
  s->pw_ready = false;  // a failed build leaves no vectors to start from
  if (warm) {
    if (!s->build_warm)
      TOPO_TRY(capture(s, &s->build_warm, &s->build_warm_kernels,
                       [&]() { return enqueue_build(s, true); }));
    TOPO_TRY(launch_graph(s, s->build_warm, s->build_warm_kernels));
  } else {
    if (!s->build)
      TOPO_TRY(capture(s, &s->build, &s->build_kernels, [&]() { return enqueue_build(s); }));
    TOPO_TRY(launch_graph(s, s->build, s->build_kernels));
  }
  int info_h[2] = {0, 0};
  TOPO_CUDA(cudaMemcpyAsync(info_h, s->info, 2 * sizeof(int), cudaMemcpyDeviceToHost, s->st));
  TOPO_CUDA(cudaStreamSynchronize(s->st));
  if (info_h[1]) {
    set_error("topo_set_density: densities must be finite and > 0");
    return TOPO_E_INVALID_ARG;
  }
  if (info_h[0]) {
    set_error("coarsest operator is not positive definite (pivot " + std::to_string(info_h[0]) + ")");
    return TOPO_E_BREAKDOWN;
  }
  s->pw_ready = s->pw_vec != nullptr;
  return TOPO_OK;
}

}  // namespace

extern "C" {

const char* topo_last_error(void) { return g_last_error.c_str(); }

topo_status topo_element_stiffness(int dim, double E, double nu, double* K0_out) {
  if ((dim != 2 && dim != 3) || !K0_out || !(E > 0.0) || !(nu > -1.0 && nu < 0.5)) {
    set_error("topo_element_stiffness: dim must be 2 or 3, E > 0, -1 < nu < 1/2");
    return TOPO_E_INVALID_ARG;
  }
  element_stiffness_host(dim, E, nu, K0_out);
  return TOPO_OK;
}

topo_status topo_solver_destroy(topo_solver* s) {
  if (!s) return TOPO_OK;
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->loop) cudaGraphExecDestroy(s->loop);
  for (int k = 0; k < 2; ++k)
    if (s->setup[k]) cudaGraphExecDestroy(s->setup[k]);
  if (s->build) cudaGraphExecDestroy(s->build);
  if (s->build_warm) cudaGraphExecDestroy(s->build_warm);
  for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
  for (void* p : s->allocs) cudaFree(p);
  if (s->sc_host) cudaFreeHost(s->sc_host);
  if (s->dots_host) cudaFreeHost(s->dots_host);
  if (s->ev_in) cudaEventDestroy(s->ev_in);
  if (s->ev_out) cudaEventDestroy(s->ev_out);
  if (s->ev_t0) cudaEventDestroy(s->ev_t0);
  if (s->ev_t1) cudaEventDestroy(s->ev_t1);
  if (s->ev_copy_in) cudaEventDestroy(s->ev_copy_in);
  if (s->ev_copy) cudaEventDestroy(s->ev_copy);
  if (s->st_copy) cudaStreamDestroy(s->st_copy);
  if (s->st) cudaStreamDestroy(s->st);
  delete s;
  return TOPO_OK;
}

static topo_status create_impl(const topo_solver_desc* d, topo_solver* s, bool arrow) {
  s->desc = *d;
  s->arrow = arrow;
  s->dim = d->dim;
  s->nlev = d->levels;
  s->prec = d->precision;
  s->nrhs = d->nrhs;
  s->ne = d->dim == 2 ? 8 : 24;
  TOPO_CUDA(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
  TOPO_CUDA(cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming));
  TOPO_CUDA(cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming));
  TOPO_CUDA(cudaEventCreate(&s->ev_t0));
  TOPO_CUDA(cudaEventCreate(&s->ev_t1));
  TOPO_CUDA(cudaStreamCreateWithFlags(&s->st_copy, cudaStreamNonBlocking));
  TOPO_CUDA(cudaEventCreateWithFlags(&s->ev_copy_in, cudaEventDisableTiming));
  TOPO_CUDA(cudaEventCreateWithFlags(&s->ev_copy, cudaEventDisableTiming));
  const int ne = s->ne, nrhs = s->nrhs;
  // element data
  std::vector<double> K0, C;
  descriptor_K0(d, K0);
  child_matrices(s->dim, K0.data(), C);
  std::vector<double> C2;
  if (!arrow && s->nlev >= 3) grandchild_matrices(s->dim, K0.data(), C2);
  s->q1_ok = (s->dim == 2) && !d->generic_kernels &&
             (d->K0 ? q1_coefficients_from_K0(K0.data(), s->q1)
                    : q1_coefficients(d->E, d->nu, K0.data(), s->q1));
  // TOPO_Q1_NARROW=1 keeps the one-column-per-lane FP32 sweeps (a reference for the two-column
  // ones, which give the same outputs)
  {
    const char* nv = std::getenv("TOPO_Q1_NARROW");
    s->q1_wide = !(nv && nv[0] == '1');
  }
  {  // TOPO_COARSE_PROLONG=0: separate prolongation and sweep kernels on the stored-matrix levels
    const char* cp = std::getenv("TOPO_COARSE_PROLONG");
    s->coarse_prolong = !(cp && cp[0] == '0');
  }
  s->hex_ok = (s->dim == 3) && !arrow && !d->generic_kernels && hex_coefficients(K0.data(), s->hex);
  s->hex_buffered = s->hex_ok && hex_buffered_env();
  s->hex_sweep = (s->dim == 3 && !arrow) ? hex_sweep_env(s->hex_ok) : 0;
  if (s->dim == 3) TOPO_CUDA(prepare_hex_tile_kernels());
  s->l1_free = (s->dim == 2) && !arrow && s->prec == TOPO_MIXED && s->nlev >= 3 &&
               !d->generic_kernels;
  // The V-cycle of a mixed solver reads FP32 coarse matrices only, so they are computed in FP32
  // (Galerkin products of FP32 inputs) unless a build-time power iteration needs FP64 operators;
  // the coarsest matrix is still accumulated and factored in FP64.
  s->h32 = !arrow && s->prec == TOPO_MIXED && d->smoother == 0 && !d->omega_auto;
  if (s->dim == 2) {
    s->C_host = C;
    s->C2_host = C2;
  }
  std::vector<float> K0f(K0.begin(), K0.end()), C32(C.begin(), C.end());
  TOPO_TRY(s->alloc(&s->K0, ne * ne));
  TOPO_TRY(s->alloc(&s->K0f, ne * ne));
  TOPO_TRY(s->alloc(&s->C, C.size()));
  TOPO_TRY(s->alloc(&s->C32, C32.size()));
  if (!C2.empty()) {
    TOPO_TRY(s->alloc(&s->C2, C2.size()));
    TOPO_CUDA(cudaMemcpy(s->C2, C2.data(), sizeof(double) * C2.size(), cudaMemcpyHostToDevice));
    if (s->h32) {
      std::vector<float> C2f(C2.begin(), C2.end());
      TOPO_TRY(s->alloc(&s->C2f, C2f.size()));
      TOPO_CUDA(cudaMemcpy(s->C2f, C2f.data(), sizeof(float) * C2f.size(), cudaMemcpyHostToDevice));
    }
  }
  TOPO_CUDA(cudaMemcpy(s->K0, K0.data(), sizeof(double) * ne * ne, cudaMemcpyHostToDevice));
  TOPO_CUDA(cudaMemcpy(s->K0f, K0f.data(), sizeof(float) * ne * ne, cudaMemcpyHostToDevice));
  TOPO_CUDA(cudaMemcpy(s->C, C.data(), sizeof(double) * C.size(), cudaMemcpyHostToDevice));
  TOPO_CUDA(cudaMemcpy(s->C32, C32.data(), sizeof(float) * C32.size(), cudaMemcpyHostToDevice));
  // levels and masks
  Dims d0{d->nx, d->ny, d->dim == 3 ? d->nz : 1, d->dim};
  s->L.resize(s->nlev);
  std::vector<uint8_t> mask((size_t)d0.dofs());
  for (long long i = 0; i < d0.dofs(); ++i) mask[i] = d->fixed[i] ? 1 : 0;
  s->fixed_host = mask;
  Dims dk = d0;
  const size_t vbytes = s->prec == TOPO_MIXED ? sizeof(float) : sizeof(double);
  for (int k = 0; k < s->nlev; ++k) {
    Level& lv = s->L[k];
    lv.d = dk;
    lv.n = dk.dofs();
    lv.m = dk.elems();
    TOPO_TRY(s->alloc(&lv.fixed, lv.n));
    TOPO_CUDA(cudaMemcpy(lv.fixed, mask.data(), lv.n, cudaMemcpyHostToDevice));
    const bool coarsest = (k == s->nlev - 1);
    const long long vl = lv.n + (arrow ? 2 : 0);
    if (k >= 1) {
      const bool l1_matrix_free = (k == 1 && s->l1_free);
      // FP32 hierarchy: FP64 matrices on the coarsest level only
      if (!l1_matrix_free && (!s->h32 || coarsest)) TOPO_TRY(s->alloc(&lv.Ae, lv.m * ne * ne));
      if (s->prec == TOPO_MIXED && !coarsest && !l1_matrix_free)
        TOPO_TRY(s->alloc(&lv.Ae32, lv.m * ne * ne));
      // element-major copy for the single-block deep tail (a level it may start at or cover)
      if (aem_level(s->dim, arrow, coarsest, l1_matrix_free, dk.nodes()))
        TOPO_TRY(s->alloc((char**)&lv.Aem, vbytes * lv.m * kAemStride));
    }
    if (arrow) {
      TOPO_TRY(s->alloc(&lv.w, lv.n));
      if (s->prec == TOPO_MIXED) TOPO_TRY(s->alloc(&lv.w32, lv.n));
    }
    if (!coarsest) {
      TOPO_TRY(s->alloc(&lv.invd, lv.n));
      if (s->prec == TOPO_MIXED) TOPO_TRY(s->alloc(&lv.invd32, lv.n));
      if (d->smoother == 1 && !arrow) {
        TOPO_TRY(s->alloc(&lv.lam_dev, 1));
        TOPO_TRY(s->alloc((char**)&lv.cd, vbytes * vl * nrhs));
      } else if (d->omega_auto && (arrow || k >= 1)) {
        TOPO_TRY(s->alloc(&lv.omega_dev, 1));
      }
      TOPO_TRY(s->alloc((char**)&lv.t, vbytes * vl * nrhs));
    }
    if (k >= 1) TOPO_TRY(s->alloc((char**)&lv.b, vbytes * vl * nrhs));
    TOPO_TRY(s->alloc((char**)&lv.z, vbytes * vl * nrhs));
    if (!coarsest) {
      std::vector<uint8_t> next;
      std::string why;
      if (!coarsen_mask(dk, mask, next, why)) {
        set_error(why);
        return TOPO_E_INVALID_ARG;
      }
      mask.swap(next);
      dk = Dims{dk.nx / 2, dk.ny / 2, dk.dim == 3 ? dk.nz / 2 : 1, dk.dim};
    }
  }
  if (s->dim == 2 && s->q1_ok && !arrow && s->prec == TOPO_MIXED) {
    // the finest mask as node pairs with an even row stride, for the FP32 two-column sweeps
    const int nx = d->nx, ny = d->ny, rsp = nx + 2;
    std::vector<uint8_t> pad((size_t)(ny + 1) * rsp * 2, 0);
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i <= nx; ++i)
        for (int c = 0; c < 2; ++c)
          pad[((size_t)j * rsp + i) * 2 + c] = s->fixed_host[((size_t)j * (nx + 1) + i) * 2 + c];
    TOPO_TRY(s->alloc(&s->fixed_pad, pad.size() / 4));
    TOPO_CUDA(cudaMemcpy(s->fixed_pad, pad.data(), pad.size(), cudaMemcpyHostToDevice));
  }
  Level& lc = s->L[s->nlev - 1];
  s->nc = (int)lc.n;
  const size_t na = (size_t)s->nc + (arrow ? 1 : 0);
  TOPO_CUDA(prepare_coarse_kernels((int)na));
  s->tail_ok = prepare_tail_kernels() == cudaSuccess;  // a cluster of the fused kernel fits
  cudaGetLastError();
  TOPO_TRY(s->alloc(&s->Adense, na * na));
  TOPO_TRY(s->alloc(&s->Ainv, na * na));
  if (s->prec == TOPO_MIXED) TOPO_TRY(s->alloc(&s->AinvDF, na * na));
  TOPO_TRY(s->alloc(&s->info, 4));
  // Newton-Schulz products (small K systems) or the block Gauss-Jordan workspace (larger ones)
  if ((!arrow || na > 128) && coarse_scratch_doubles((int)na))
    TOPO_TRY(s->alloc(&s->Ascratch, coarse_scratch_doubles((int)na)));
  TOPO_TRY(s->alloc(&s->pw_est, 2));
  {  // power-iteration vectors (with the trailing lambda entry of IP systems, padded to even)
    size_t tot = 0;
    s->pw_off.assign(s->nlev, 0);
    for (int k = 0; k < s->nlev; ++k) {
      s->pw_off[k] = tot;
      if (s->L[k].omega_dev || s->L[k].lam_dev) tot += (size_t)s->L[k].n + 2;
    }
    s->pw_len = tot;
    if (tot) TOPO_TRY(s->alloc(&s->pw_vec, tot));
  }
  // densities and CG vectors (IP systems: trailing lambda entry, padded to an even length)
  const long long m = s->L[0].m;
  const long long n = s->L[0].n + (arrow ? 2 : 0);
  TOPO_TRY(s->alloc(&s->x, m));
  if (s->hex_buffered) TOPO_TRY(s->alloc(&s->hexR, (size_t)m * 24 * nrhs));
  if ((s->q1_ok || s->hex_ok) && !arrow) {  // pair-arithmetic outer operator: default for mixed
    TOPO_TRY(s->alloc(&s->xdf, m));
    s->outer_df = s->prec == TOPO_MIXED ? 1 : 0;
  }
  if (arrow) s->outer_df = s->prec == TOPO_MIXED ? 1 : 0;  // the Z node pass in pairs
  if (s->prec == TOPO_MIXED) {
    TOPO_TRY(s->alloc(&s->x32, m));
    TOPO_TRY(s->alloc((float**)&s->rv, n * nrhs));
  }
  if (arrow) {
    TOPO_TRY(s->alloc(&s->se, m));
    if (s->prec == TOPO_MIXED) {
      TOPO_TRY(s->alloc(&s->se32, m));
      TOPO_TRY(s->alloc(&s->g32, m * ne));
      TOPO_TRY(s->alloc(&s->Dinv32, m));
    }
  }
  TOPO_TRY(s->alloc(&s->bbuf, n * nrhs));
  TOPO_TRY(s->alloc(&s->z, n * nrhs));
  TOPO_TRY(s->alloc(&s->r, n * nrhs));
  TOPO_TRY(s->alloc(&s->p, n * nrhs));
  TOPO_TRY(s->alloc(&s->q, n * nrhs));
  if (d->flexible) TOPO_TRY(s->alloc((char**)&s->yold, vbytes * n * nrhs));
  // per-block partials: fixed-grid reductions write up to kMaxRedValues values per block
  // (kRedBlocks blocks); the node-parallel fused operator writes one per block
  const long long pb = std::max<long long>((long long)kMaxRedValues * kRedBlocks,
                                           blocks_for(s->L[0].d.nodes()));
  TOPO_TRY(s->alloc(&s->partials, pb * nrhs));
  TOPO_TRY(s->alloc(&s->counters, nrhs));
  TOPO_CUDA(cudaMemset(s->counters, 0, sizeof(unsigned) * nrhs));
  TOPO_TRY(s->alloc(&s->sc, nrhs));
  TOPO_CUDA(cudaMemset(s->sc, 0, sizeof(CgScalars) * nrhs));
  TOPO_TRY(s->alloc(&s->dots, nrhs));
  TOPO_CUDA(cudaMallocHost((void**)&s->sc_host, sizeof(CgScalars) * nrhs));
  TOPO_CUDA(cudaMallocHost((void**)&s->dots_host, sizeof(double) * nrhs));
  s->prof_ev.resize(2 * s->graph_iters * topo_solver::kProfKinds);
  for (auto& e : s->prof_ev) TOPO_CUDA(cudaEventCreate(&e));
  TOPO_CUDA(cudaDeviceSynchronize());
  return TOPO_OK;
}

// Descriptor checks shared by topo_solver_create, topo_solver_workspace_bytes and the IP / OC
// drivers (what names the caller in the messages).
topo_status validate_desc(const topo_solver_desc* d, const char* what) {
  const std::string w(what);
  if (!d || !d->fixed) {
    set_error(w + ": null argument");
    return TOPO_E_INVALID_ARG;
  }
  if ((d->dim != 2 && d->dim != 3) || d->nx < 1 || d->ny < 1 || (d->dim == 3 && d->nz < 1) ||
      d->levels < 1 || d->levels > 16 || (d->precision != TOPO_FP64 && d->precision != TOPO_MIXED) ||
      d->nu1 < 0 || d->nu2 < 0 || !(d->omega > 0.0 && d->omega <= 1.0) || d->max_iter < 0 ||
      d->nrhs < 1 || d->nrhs > kMaxRhs || !(d->E > 0.0) || !(d->nu > -1.0 && d->nu < 0.5) ||
      (d->smoother != 0 && d->smoother != 1)) {
    set_error(w + ": invalid descriptor field");
    return TOPO_E_INVALID_ARG;
  }
  if (d->K0) {
    const int ne = d->dim == 2 ? 8 : 24;
    double mx = 0.0;
    for (int i = 0; i < ne * ne; ++i) {
      if (!std::isfinite(d->K0[i])) {
        set_error(w + ": K0 has a non-finite entry");
        return TOPO_E_INVALID_ARG;
      }
      mx = std::max(mx, std::fabs(d->K0[i]));
    }
    for (int i = 0; i < ne; ++i)
      for (int j = 0; j < i; ++j)
        if (std::fabs(d->K0[i * ne + j] - d->K0[j * ne + i]) > 1e-12 * mx) {
          set_error(w + ": K0 is not symmetric");
          return TOPO_E_INVALID_ARG;
        }
    if (!(mx > 0.0)) {
      set_error(w + ": K0 is zero");
      return TOPO_E_INVALID_ARG;
    }
  }
  const Dims dfine{d->nx, d->ny, d->dim == 3 ? d->nz : 1, d->dim};
  if (dfine.dofs() >= (1LL << 31)) {  // kernels index nodes and DOFs with 32-bit arithmetic
    set_error(w + ": grid has 2^31 or more DOFs");
    return TOPO_E_INVALID_ARG;
  }
  const int f = 1 << (d->levels - 1);
  if (d->nx % f || d->ny % f || (d->dim == 3 && d->nz % f)) {
    set_error(w + ": grid not divisible by 2^(levels-1)");
    return TOPO_E_INVALID_ARG;
  }
  Dims dc{d->nx / f, d->ny / f, d->dim == 3 ? d->nz / f : 1, d->dim};
  if (dc.dofs() > 4096) {
    set_error(w + ": coarsest level has more than 4096 DOFs; use more levels");
    return TOPO_E_INVALID_ARG;
  }
  return TOPO_OK;
}

// Device bytes create_impl allocates for d (the same decisions in the same order, counted on the
// host).  Masks incompatible with coarsening are rejected as create_impl does.
topo_status plan_bytes(const topo_solver_desc* d, bool arrow, size_t* out) {
  const int dim = d->dim, ne = dim == 2 ? 8 : 24, nrhs = d->nrhs, nlev = d->levels;
  const bool mixed = d->precision == TOPO_MIXED;
  size_t bytes = 0;
  auto add = [&](size_t count, size_t elem) { bytes += std::max<size_t>(count, 1) * elem; };
  std::vector<double> K0, C, C2;
  descriptor_K0(d, K0);
  child_matrices(dim, K0.data(), C);
  if (!arrow && nlev >= 3) grandchild_matrices(dim, K0.data(), C2);
  Q1Coef q1;
  HexCoef hex;
  const bool q1_ok = dim == 2 && !d->generic_kernels &&
                     (d->K0 ? q1_coefficients_from_K0(K0.data(), q1)
                            : q1_coefficients(d->E, d->nu, K0.data(), q1));
  const bool hex_ok = dim == 3 && !arrow && !d->generic_kernels && hex_coefficients(K0.data(), hex);
  const bool l1_free = dim == 2 && !arrow && mixed && nlev >= 3 && !d->generic_kernels;
  const bool h32 = !arrow && mixed && d->smoother == 0 && !d->omega_auto;
  add(ne * ne, sizeof(double));
  add(ne * ne, sizeof(float));
  add(C.size(), sizeof(double));
  add(C.size(), sizeof(float));
  if (!C2.empty()) {
    add(C2.size(), sizeof(double));
    if (h32) add(C2.size(), sizeof(float));
  }
  Dims dk{d->nx, d->ny, dim == 3 ? d->nz : 1, dim};
  std::vector<uint8_t> mask((size_t)dk.dofs());
  for (size_t i = 0; i < mask.size(); ++i) mask[i] = d->fixed[i] ? 1 : 0;
  const size_t vbytes = mixed ? sizeof(float) : sizeof(double);
  std::vector<long long> lev_n(nlev);
  std::vector<bool> pw_level(nlev, false);
  long long nc = 0;
  for (int k = 0; k < nlev; ++k) {
    const long long n = dk.dofs(), m = dk.elems();
    lev_n[k] = n;
    add(n, 1);
    const bool coarsest = k == nlev - 1;
    const long long vl = n + (arrow ? 2 : 0);
    if (k >= 1) {
      const bool l1_matrix_free = k == 1 && l1_free;
      if (!l1_matrix_free && (!h32 || coarsest)) add(m * ne * ne, sizeof(double));
      if (mixed && !coarsest && !l1_matrix_free) add(m * ne * ne, sizeof(float));
      if (aem_level(dim, arrow, coarsest, l1_matrix_free, dk.nodes())) add(vbytes * m * kAemStride, 1);
    }
    if (arrow) {
      add(n, sizeof(double));
      if (mixed) add(n, sizeof(float));
    }
    if (!coarsest) {
      add(n, sizeof(double));
      if (mixed) add(n, sizeof(float));
      if (d->smoother == 1 && !arrow) {
        add(1, sizeof(double));
        add(vbytes * vl * nrhs, 1);
        pw_level[k] = true;
      } else if (d->omega_auto && (arrow || k >= 1)) {
        add(1, sizeof(double));
        pw_level[k] = true;
      }
      add(vbytes * vl * nrhs, 1);
    }
    if (k >= 1) add(vbytes * vl * nrhs, 1);
    add(vbytes * vl * nrhs, 1);
    if (!coarsest) {
      std::vector<uint8_t> next;
      std::string why;
      if (!coarsen_mask(dk, mask, next, why)) {
        set_error(why);
        return TOPO_E_INVALID_ARG;
      }
      mask.swap(next);
      dk = Dims{dk.nx / 2, dk.ny / 2, dk.dim == 3 ? dk.nz / 2 : 1, dk.dim};
    } else {
      nc = n;
    }
  }
  if (dim == 2 && q1_ok && !arrow && mixed)
    add((size_t)(d->ny + 1) * (d->nx + 2) * 2 / 4, sizeof(unsigned));
  const size_t na = (size_t)nc + (arrow ? 1 : 0);
  add(na * na, sizeof(double));
  add(na * na, sizeof(double));
  if (mixed) add(na * na, sizeof(float2));
  add(4, sizeof(int));
  if ((!arrow || na > 128) && coarse_scratch_doubles((int)na))
    add(coarse_scratch_doubles((int)na), sizeof(double));
  add(2, sizeof(double));
  size_t tot = 0;
  for (int k = 0; k < nlev; ++k)
    if (pw_level[k]) tot += (size_t)lev_n[k] + 2;
  if (tot) add(tot, sizeof(double));
  const Dims d0{d->nx, d->ny, dim == 3 ? d->nz : 1, dim};
  const long long m = d0.elems();
  const long long n = d0.dofs() + (arrow ? 2 : 0);
  add(m, sizeof(double));
  if (hex_ok && hex_buffered_env()) add((size_t)m * 24 * nrhs, sizeof(double));
  if ((q1_ok || hex_ok) && !arrow) add(m, sizeof(float2));
  if (mixed) {
    add(m, sizeof(float));
    add(n * nrhs, sizeof(float));
  }
  if (arrow) {
    add(m, sizeof(double));
    if (mixed) {
      add(m, sizeof(float));
      add(m * ne, sizeof(float));
      add(m, sizeof(float));
    }
  }
  for (int v = 0; v < 5; ++v) add(n * nrhs, sizeof(double));
  if (d->flexible) add(vbytes * n * nrhs, 1);
  const long long pb = std::max<long long>((long long)kMaxRedValues * kRedBlocks,
                                           blocks_for(d0.nodes()));
  add(pb * nrhs, sizeof(double));
  add(nrhs, sizeof(unsigned));
  add(nrhs, sizeof(CgScalars));
  add(nrhs, sizeof(double));
  *out = bytes;
  return TOPO_OK;
}

topo_status topo_solver_workspace_bytes(const topo_solver_desc* d, size_t* bytes) {
  TOPO_TRY(validate_desc(d, "topo_solver_workspace_bytes"));
  if (!bytes) {
    set_error("topo_solver_workspace_bytes: null argument");
    return TOPO_E_INVALID_ARG;
  }
  return plan_bytes(d, false, bytes);
}

topo_status topo_solver_create(const topo_solver_desc* d, topo_solver** out) {
  if (!out) {
    set_error("topo_solver_create: null argument");
    return TOPO_E_INVALID_ARG;
  }
  *out = nullptr;
  TOPO_TRY(validate_desc(d, "topo_solver_create"));
  topo_solver* s = new topo_solver();
  topo_status st = create_impl(d, s, false);
  if (st != TOPO_OK) {
    std::string keep = g_last_error;
    topo_solver_destroy(s);
    g_last_error = keep;
    return st;
  }
  *out = s;
  return TOPO_OK;
}

topo_status topo_set_outer_precision(topo_solver* s, int mode) {
  if (!s || (mode != 0 && mode != 1)) {
    set_error("topo_set_outer_precision: null solver or mode not 0/1");
    return TOPO_E_INVALID_ARG;
  }
  const int want = (mode == 1 && s->xdf) ? 1 : 0;
  if (want != s->outer_df) {
    s->outer_df = want;
    if (s->graph) {  // captured iterations hold the old kernel
      cudaGraphExecDestroy(s->graph);
      s->graph = nullptr;
    }
    if (s->loop) {
      cudaGraphExecDestroy(s->loop);
      s->loop = nullptr;
    }
  }
  return TOPO_OK;
}

// Captured graphs hold the V-cycle's kernels and launch shapes: drop them after a change.
void drop_graphs(topo_solver* s) {
  for (int u = 0; u < 2; ++u)
    if (s->setup[u]) {
      cudaGraphExecDestroy(s->setup[u]);
      s->setup[u] = nullptr;
    }
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  if (s->loop) {
    cudaGraphExecDestroy(s->loop);
    s->loop = nullptr;
  }
}

topo_status topo_set_vcycle_fusion(topo_solver* s, int on) {
  if (!s) {
    set_error("topo_set_vcycle_fusion: null solver");
    return TOPO_E_INVALID_ARG;
  }
  const bool want = on != 0;
  if (want != s->fuse_on) {
    s->fuse_on = want;
    drop_graphs(s);
  }
  return TOPO_OK;
}

topo_status topo_set_wait_limit_ns(topo_solver* s, unsigned long long ns) {
  if (!s) {
    set_error("topo_set_wait_limit_ns: null solver");
    return TOPO_E_INVALID_ARG;
  }
  if (ns != s->wait_ns) {
    s->wait_ns = ns;
    drop_graphs(s);
  }
  return TOPO_OK;
}

topo_status topo_set_sweep_rows(topo_solver* s, int rows) {
  if (!s || rows < 0 || rows > 32 || rows == 1) {
    set_error("topo_set_sweep_rows: null solver or rows outside {0} and 2..32");
    return TOPO_E_INVALID_ARG;
  }
  if (rows != s->sweep_rows) {
    s->sweep_rows = rows;
    drop_graphs(s);
  }
  return TOPO_OK;
}

topo_status topo_set_graph_mode(topo_solver* s, int mode) {
  if (!s || (mode != 0 && mode != 1)) {
    set_error("topo_set_graph_mode: null solver or mode not 0/1");
    return TOPO_E_INVALID_ARG;
  }
  s->graph_mode = mode;
  return TOPO_OK;
}

topo_status topo_set_stream(topo_solver* s, void* stream) {
  if (!s) return TOPO_E_INVALID_ARG;
  s->user = (cudaStream_t)stream;
  return TOPO_OK;
}

size_t topo_solver_device_bytes(const topo_solver* s) { return s ? s->bytes : 0; }

unsigned long long topo_solver_launch_count(const topo_solver* s) { return s ? s->launches : 0; }

topo_status topo_set_profiling(topo_solver* s, int on) {
  return topo_set_profiling_mask(s, on ? 1u : 0u);
}

topo_status topo_set_profiling_mask(topo_solver* s, unsigned mask) {
  if (!s || mask >= (1u << topo_solver::kProfKinds)) {
    set_error("topo_set_profiling_mask: null solver or mask beyond the profiled kinds");
    return TOPO_E_INVALID_ARG;
  }
  if (mask != s->prof_mask) {
    s->prof_mask = mask;
    s->profiling = mask != 0;
    if (s->graph) {  // the iteration graph gains or loses event nodes
      cudaGraphExecDestroy(s->graph);
      s->graph = nullptr;
    }
  }
  for (int k = 0; k < topo_solver::kProfKinds; ++k) {
    s->prof_ms[k] = 0.0;
    s->prof_count[k] = 0;
  }
  return TOPO_OK;
}

topo_status topo_get_profile(const topo_solver* s, double* operator_ms_total, long long* count) {
  return topo_get_profile_kernel(s, 0, operator_ms_total, count);
}

topo_status topo_get_profile_kernel(const topo_solver* s, int kind, double* ms_total,
                                    long long* count) {
  if (!s || !ms_total || !count || kind < 0 || kind >= topo_solver::kProfKinds) {
    set_error("topo_get_profile_kernel: null argument or kind outside 0..11");
    return TOPO_E_INVALID_ARG;
  }
  *ms_total = s->prof_ms[kind];
  *count = s->prof_count[kind];
  return TOPO_OK;
}

int topo_level_elems(const topo_solver* s, int level) {
  if (!s || level < 0 || level >= s->nlev) return -1;
  return (int)s->L[level].m;
}

topo_status topo_set_density(topo_solver* s, const double* x) {
  if (!s || !x) {
    set_error("topo_set_density: null argument");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard g(s);
  const long long m = s->L[0].m;
  TOPO_CUDA(cudaMemcpyAsync(s->x, x, sizeof(double) * m, cudaMemcpyDeviceToDevice, s->st));
  topo_status st = build_hierarchy(s);
  s->have_density = (st == TOPO_OK);
  return st;
}

// One JSON line per solve (topo_set_record_file): the configuration, the outcome and the rate.
void append_record(const topo_solver* s, double tol, const topo_solve_info& in, topo_status st) {
  if (s->record_path.empty()) return;
  FILE* fp = std::fopen(s->record_path.c_str(), "a");
  if (!fp) return;
  long long nfree = 0;
  for (uint8_t f : s->fixed_host) nfree += f ? 0 : 1;
  const double rate = in.wall_ms > 0.0 ? (double)nfree * in.iterations / (in.wall_ms * 1e-3) : 0.0;
  std::fprintf(fp,
               "{\"call\": \"solve\", \"system\": \"%s\", \"dim\": %d, \"nx\": %d, \"ny\": %d, "
               "\"nz\": %d, \"levels\": %d, \"precision\": \"%s\", \"smoother\": \"%s\", "
               "\"nu1\": %d, \"nu2\": %d, \"omega\": %.17g, \"nrhs\": %d, \"free_dofs\": %lld, "
               "\"tol\": %.17g, \"iterations\": %d, \"rel_residual\": %.17g, \"wall_ms\": %.6f, "
               "\"dof_it_per_s\": %.6g, \"status\": %d}\n",
               s->arrow ? "Z" : "K", s->dim, s->desc.nx, s->desc.ny, s->dim == 3 ? s->desc.nz : 0,
               s->nlev, s->prec == TOPO_MIXED ? "mixed" : "fp64",
               s->desc.smoother == 1 ? "chebyshev" : "jacobi", s->desc.nu1, s->desc.nu2,
               s->desc.omega, s->nrhs, nfree, tol, in.iterations, in.rel_residual, in.wall_ms, rate,
               (int)st);
  std::fclose(fp);
}

topo_status topo_solve(topo_solver* s, const double* b, double* u, double tol, int use_x0,
                       topo_solve_info* info) {
  if (!s || !b || !u || !(tol >= 0.0)) {
    set_error("topo_solve: invalid argument");
    return TOPO_E_INVALID_ARG;
  }
  if (!s->have_density) {
    set_error("topo_solve: call topo_set_density first");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard g(s);
  topo_solve_info local{};
  topo_solve_info* out = info ? info : &local;
  const topo_status st = bounds_status(
      s->prec == TOPO_MIXED ? solve_impl<float>(s, b, u, tol, use_x0, out)
                            : solve_impl<double>(s, b, u, tol, use_x0, out),
      "topo_solve");
  append_record(s, tol, *out, st);
  return st;
}

topo_status topo_set_record_file(topo_solver* s, const char* path) {
  if (!s) {
    set_error("topo_set_record_file: null solver");
    return TOPO_E_INVALID_ARG;
  }
  s->record_path = path ? path : "";
  return TOPO_OK;
}

topo_status topo_solve_host(topo_solver* s, const double* x, const double* b, double* u,
                            double tol, topo_solve_info* info) {
  if (!s || !x || !b || !u || !(tol >= 0.0)) {
    set_error("topo_solve_host: invalid argument");
    return TOPO_E_INVALID_ARG;
  }
  if (s->arrow) {
    set_error("topo_solve_host: K systems only");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard g(s);
  const long long m = s->L[0].m, n = s->L[0].n * s->nrhs;
  // b travels on the copy stream (after the solver's earlier work on its buffer) while the
  // hierarchy is built from x
  TOPO_CUDA(cudaEventRecord(s->ev_copy_in, s->st));
  TOPO_CUDA(cudaStreamWaitEvent(s->st_copy, s->ev_copy_in, 0));
  TOPO_CUDA(cudaMemcpyAsync(s->bbuf, b, sizeof(double) * n, cudaMemcpyHostToDevice, s->st_copy));
  TOPO_CUDA(cudaEventRecord(s->ev_copy, s->st_copy));
  TOPO_CUDA(cudaMemcpyAsync(s->x, x, sizeof(double) * m, cudaMemcpyHostToDevice, s->st));
  topo_status st = build_hierarchy(s);
  s->have_density = (st == TOPO_OK);
  if (st != TOPO_OK) {
    cudaStreamSynchronize(s->st_copy);
    return st;
  }
  TOPO_CUDA(cudaStreamWaitEvent(s->st, s->ev_copy, 0));
  st = s->prec == TOPO_MIXED ? solve_impl<float>(s, s->bbuf, s->z, tol, 0, info)
                             : solve_impl<double>(s, s->bbuf, s->z, tol, 0, info);
  if (st != TOPO_OK && st != TOPO_E_NOT_CONVERGED) return st;
  TOPO_CUDA(cudaMemcpyAsync(u, s->z, sizeof(double) * n, cudaMemcpyDeviceToHost, s->st));
  TOPO_CUDA(cudaStreamSynchronize(s->st));
  return bounds_status(st, "topo_solve_host");
}

topo_status topo_apply_K(topo_solver* s, const double* v, double* y) {
  if (!s || !v || !y || !s->have_density) {
    set_error("topo_apply_K: invalid argument or no density set");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard g(s);
  return bounds_status(apply_outer(s, v, y, nullptr), "topo_apply_K");
}

int topo_bounds_check_enabled(void) {
#ifdef TOPO_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

topo_status topo_bounds_report(unsigned long long* count, long long* index, long long* size,
                               char* file, int file_len, int* line, int reset) {
  unsigned long long c = 0;
  BoundsRecord rec{};
  const char* f = "";
  const cudaError_t e = read_bounds(&c, &rec, &f, reset != 0);
  if (e != cudaSuccess) return cuda_status(e, "topo_bounds_report");
  if (count) *count = c;
  if (index) *index = rec.index;
  if (size) *size = rec.size;
  if (line) *line = rec.line;
  if (file && file_len > 0) {
    std::strncpy(file, f, (size_t)file_len - 1);
    file[file_len - 1] = '\0';
  }
  return TOPO_OK;
}

topo_status topo_bounds_selftest(long long i, long long n) {
#ifdef TOPO_BOUNDS_CHECK
  int* out = nullptr;
  TOPO_CUDA(cudaMalloc(&out, sizeof(int)));
  k_bounds_selftest<<<1, 1>>>(i, n, out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(out);
  if (e != cudaSuccess) return cuda_status(e, "topo_bounds_selftest");
  return TOPO_OK;
#else
  (void)i;
  (void)n;
  set_error("topo_bounds_selftest: this library was built without TOPO_BOUNDS_CHECK");
  return TOPO_E_INVALID_ARG;
#endif
}

topo_status topo_check_conversions(const double* d, const float* f, long long n,
                                   unsigned long long* mismatches) {
  if (n < 0 || !mismatches || (n > 0 && (!d || !f))) {
    set_error("topo_check_conversions: invalid argument");
    return TOPO_E_INVALID_ARG;
  }
  unsigned long long* bad = nullptr;
  TOPO_CUDA(cudaMalloc(&bad, 2 * sizeof(unsigned long long)));
  cudaError_t e = cudaMemset(bad, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess && n > 0) e = launch_check_conversions(d, f, n, bad, nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpy(mismatches, bad, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  cudaFree(bad);
  if (e != cudaSuccess) return cuda_status(e, "topo_check_conversions");
  return TOPO_OK;
}

topo_status topo_apply_vcycle(topo_solver* s, const double* r, double* y) {
  if (!s || !r || !y || !s->have_density) {
    set_error("topo_apply_vcycle: invalid argument or no density set");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard g(s);
  const long long n = s->L[0].n * s->nrhs;
  if (s->prec == TOPO_MIXED) {
    TOPO_CUDA(launch_convert_d2f(r, (float*)s->rv, n, s->st));
    float* out = nullptr;
    TOPO_TRY(vcycle<float>(s, 0, (const float*)s->rv, &out, nullptr));
    TOPO_CUDA(launch_convert_f2d(out, y, n, s->st));
    return bounds_status(TOPO_OK, "topo_apply_vcycle");
  }
  TOPO_CUDA(cudaMemcpyAsync(s->r, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->st));
  double* out = nullptr;
  TOPO_TRY(vcycle<double>(s, 0, s->r, &out, nullptr));
  TOPO_CUDA(cudaMemcpyAsync(y, out, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->st));
  return bounds_status(TOPO_OK, "topo_apply_vcycle");
}

topo_status topo_get_level_matrices(topo_solver* s, int level, double* out_host) {
  if (!s || !out_host || level < 1 || level >= s->nlev || !s->have_density) {
    set_error("topo_get_level_matrices: level must be in [1, levels) after topo_set_density");
    return TOPO_E_INVALID_ARG;
  }
  if (!s->L[level].Ae && !s->L[level].Ae32) {
    set_error("topo_get_level_matrices: this level is applied matrix-free (mixed precision)");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard g(s);
  const Level& lv = s->L[level];
  const long long ne2 = (long long)s->ne * s->ne;
  std::vector<double> tmp(lv.m * ne2);
  if (lv.Ae) {
    TOPO_CUDA(cudaMemcpyAsync(tmp.data(), lv.Ae, sizeof(double) * tmp.size(),
                              cudaMemcpyDeviceToHost, s->st));
    TOPO_CUDA(cudaStreamSynchronize(s->st));
  } else {  // FP32 hierarchy: the stored FP32 matrices, widened
    std::vector<float> t32(tmp.size());
    TOPO_CUDA(cudaMemcpyAsync(t32.data(), lv.Ae32, sizeof(float) * t32.size(),
                              cudaMemcpyDeviceToHost, s->st));
    TOPO_CUDA(cudaStreamSynchronize(s->st));
    for (size_t q = 0; q < tmp.size(); ++q) tmp[q] = t32[q];
  }
  for (long long e = 0; e < lv.m; ++e)
    for (long long q = 0; q < ne2; ++q) out_host[e * ne2 + q] = tmp[q * lv.m + e];
  return TOPO_OK;
}

topo_status topo_compliance(topo_solver* s, const double* f, const double* u, double* c) {
  if (!s || !f || !u || !c) {
    set_error("topo_compliance: null argument");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard g(s);
  TOPO_CUDA(launch_dot(s->L[0].n, s->nrhs, f, u, s->partials, s->counters, s->dots, s->st));
  TOPO_CUDA(cudaMemcpyAsync(s->dots_host, s->dots, sizeof(double) * s->nrhs, cudaMemcpyDeviceToHost,
                            s->st));
  TOPO_CUDA(cudaStreamSynchronize(s->st));
  for (int k = 0; k < s->nrhs; ++k) c[k] = s->dots_host[k];
  return TOPO_OK;
}

topo_status topo_element_energy(topo_solver* s, const double* u, double* E) {
  if (!s || !u || !E) {
    set_error("topo_element_energy: null argument");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard g(s);
  TOPO_CUDA(launch_element_energy(s->L[0].d, s->K0, u, u, E, 1.0, s->st));
  return TOPO_OK;
}

topo_status topo_grad_x(topo_solver* s, const double* lam, const double* u, double* gx) {
  if (!s || !lam || !u || !gx) {
    set_error("topo_grad_x: null argument");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard g(s);
  TOPO_CUDA(launch_element_energy(s->L[0].d, s->K0, u, lam, gx, -1.0, s->st));
  return TOPO_OK;
}

}  // extern "C"

namespace topo {

topo_status solver_create_internal(const topo_solver_desc* d, bool arrow, topo_solver** out) {
  if (!arrow) return topo_solver_create(d, out);
  if (!out) return TOPO_E_INVALID_ARG;
  *out = nullptr;
  TOPO_TRY(validate_desc(d, "topo_solver_create"));
  topo_status st;
  if (d->nrhs != 1) {
    set_error("IP systems are solved one right-hand side at a time");
    return TOPO_E_INVALID_ARG;
  }
  topo_solver* s = new topo_solver();
  st = create_impl(d, s, true);
  if (st != TOPO_OK) {
    std::string keep = g_last_error;
    topo_solver_destroy(s);
    g_last_error = keep;
    return st;
  }
  *out = s;
  return TOPO_OK;
}

topo_status solver_build(topo_solver* s) {
  topo_status st = build_hierarchy(s);
  s->have_density = (st == TOPO_OK);
  return st;
}

topo_status solver_solve(topo_solver* s, const double* b, double* u, double tol, int use_x0,
                         topo_solve_info* info) {
  topo_solve_info local{};
  topo_solve_info* out = info ? info : &local;
  const topo_status st = bounds_status(
      s->prec == TOPO_MIXED ? solve_impl<float>(s, b, u, tol, use_x0, out)
                            : solve_impl<double>(s, b, u, tol, use_x0, out),
      "solve");
  append_record(s, tol, *out, st);
  return st;
}

}  // namespace topo
