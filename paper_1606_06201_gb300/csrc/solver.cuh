// Solver object shared by the host translation units (solver.cu: MGCG; ipoc.cu: IP and OC).
#pragma once

#include <string>
#include <vector>

#include "topo_internal.cuh"

using namespace topo;

#define TOPO_TRY(expr)            \
  do {                            \
    topo_status _s = (expr);      \
    if (_s != TOPO_OK) return _s; \
  } while (0)

struct topo_solver {
  topo_solver_desc desc{};
  int dim = 2, nlev = 1, prec = TOPO_FP64, nrhs = 1, ne = 8;
  cudaStream_t st = nullptr;     // private stream
  cudaStream_t user = nullptr;   // caller's stream (nullptr = legacy default stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  cudaStream_t st_copy = nullptr;  // host-to-device copies that overlap the hierarchy build
  cudaEvent_t ev_copy_in = nullptr, ev_copy = nullptr;
  std::vector<Level> L;
  std::vector<uint8_t> fixed_host;
  double* K0 = nullptr;
  float* K0f = nullptr;
  double* C = nullptr;           // constant child matrices P_c^T K0 P_c
  std::vector<double> C_host, C2_host;  // host copies of C and C2 (kernel-parameter tables)
  Q1Coef q1{};                   // butterfly coefficients of the 2D K0
  bool q1_ok = false;            // 2D and T^T Khat T reproduces K0: use the warp-sweep kernels
  bool q1_wide = true;           // FP32 finest sweeps with two node columns per lane (kernels_q1w.cu)
  int sweep_rows = 0;            // strip height of the 2D finest-level warp sweeps (0: automatic)
  unsigned long long wait_ns = 1000000000ull;  // bound of the device-side waits (topo_set_wait_limit_ns)
  unsigned* fixed_pad = nullptr; // 2D finest mask as node pairs, row stride (nx + 2) / 2 words
  double* x = nullptr;
  float* x32 = nullptr;
  float* C32 = nullptr;          // FP32 copy of C (matrix-free first coarse level)
  double* C2 = nullptr;          // composite matrices two levels down (second coarse level)
  float* C2f = nullptr;          // FP32 copy of C2 (FP32 hierarchy)
  bool h32 = false;              // mixed K solver with fixed damping: coarse matrices built in FP32
  bool l1_free = false;          // mixed 2D K systems: level 1 applied matrix-free in FP32
  // Arrow (IP) systems Z = [K 0; 0 0] + [B; e^T] D^{-1} [B^T e] (Eq. (nwtr2Z)): vectors carry a
  // trailing lambda entry; g_e = K0 u_e and Dinv = 1/D on the finest level are owned by the IP
  // driver; zll points to Z_ll = sum 1/D on the device.
  bool arrow = false;
  double* pw_est = nullptr;      // power-iteration scalars (adaptive damping)
  const double* g = nullptr;
  const double* Dinv = nullptr;
  const double* zll = nullptr;
  float* g32 = nullptr;
  float* Dinv32 = nullptr;
  double* se = nullptr;          // element scalars s_e of the Z operator
  // SIMP model (Sec. 9): the outer CG applies the exact Z with the filter (launch_simp_z_apply);
  // g and Dinv above then hold the hierarchy's element-local columns and weights.
  struct {
    bool on = false;
    double rmin = 0.0;
    int R = 0;
    const double* invS = nullptr;
    const double* Dinv = nullptr;  // exact 1 / D
    double* ea = nullptr;
    double* eb = nullptr;
  } simp;
  float* se32 = nullptr;
  int nc = 0;                    // DOFs of the coarsest level
  double* Adense = nullptr;
  double* Ainv = nullptr;
  float2* AinvDF = nullptr;               // Ainv as float pairs (mixed precision)
  double* Ascratch = nullptr;    // Newton-Schulz products of the coarsest inverse (small n)
  int* info = nullptr;           // [0] coarsest pivot failure, [1] bad density, [2] Newton-Schulz flag
  double *z = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
  void* yold = nullptr;          // previous preconditioned residual (flexible beta)
  void* rv = nullptr;            // residual in V-cycle precision (mixed)
  void* yv = nullptr;            // where the captured V-cycle leaves its result
  double* partials = nullptr;
  unsigned* counters = nullptr;
  CgScalars* sc = nullptr;
  CgScalars* sc_host = nullptr;  // pinned
  double* dots = nullptr;
  double* dots_host = nullptr;
  double* bbuf = nullptr;        // solver-owned copy of the right-hand side
  cudaGraphExec_t loop = nullptr;         // persistent CG: while-node over one iteration
  int loop_kernels = 0;                   // kernels per loop iteration
  double loop_tol = -1.0;
  int graph_mode = 0;                     // 0 replayed blocks of iterations, 1 while-node loop
  float2* xdf = nullptr;                  // densities as float pairs (pair-arithmetic operator)
  bool hex_ok = false;                    // 3D outer operator in the Walsh-Hadamard basis
  HexCoef hex{};
  double* hexR = nullptr;                 // its element forces (24 x elems x nrhs)
  bool hex_buffered = true;               // the two-kernel form with hexR (else the tile form)
  int hex_sweep = 0;                      // 3D finest V-cycle operator: 0 node-parallel,
                                          // 1 tile dense (same bits as 0), 2 tile Walsh-Hadamard,
                                          // 3 tile dense on the tensor cores (3 x TF32)
  bool coarse_prolong = true;             // 2D coarse levels with element matrices: prolongation
                                          // and first post-sweep in one kernel
  int outer_df = 0;                       // outer operator in float-pair arithmetic (1) or FP64
  bool tail_ok = false;                   // the fused deep-level kernel can run on this device
  bool fuse_on = true;                    // fused V-cycle kernels in use (topo_set_vcycle_fusion)
  bool no_loop = false;                   // conditional graphs unavailable on this device
  cudaGraphExec_t graph = nullptr;        // graph_iters CG iterations (profiling runs)
  int graph_kernels = 0;
  double graph_tol = -1.0;                // tolerance baked into the captured graphs
  cudaGraphExec_t setup[2] = {nullptr, nullptr};  // CG start (use_x0 = 0 / 1)
  int setup_kernels[2] = {0, 0};
  double setup_tol[2] = {-1.0, -1.0};
  cudaGraphExec_t build = nullptr;        // Galerkin hierarchy and coarsest factorisation
  int build_kernels = 0;
  cudaGraphExec_t build_warm = nullptr;   // the same with warm-started power iterations
  int build_warm_kernels = 0;
  double* pw_vec = nullptr;               // power-iteration vectors of the levels, kept
  std::vector<size_t> pw_off;             // between builds (offsets into pw_vec)
  size_t pw_len = 0;                      // doubles in pw_vec
  bool pw_ready = false;                  // pw_vec holds the last build's vectors
  int graph_iters = 4;
  unsigned long long launches = 0;        // kernels launched by this solver
  bool profiling = false;
  unsigned prof_mask = 0;                 // profiled kinds (bit k = kind k)
  // Profiling: event pairs per (kind, iteration slot) of the block graph; kinds as
  // topo_get_profile_kernel (0 outer operator, 1-4 finest-level V-cycle kernels, 5-7 V-cycle parts).
  static constexpr int kProfKinds = 12;
  std::vector<cudaEvent_t> prof_ev;
  double prof_ms[kProfKinds] = {};
  long long prof_count[kProfKinds] = {};
  int prof_slot = -1;                     // slot of the iteration being captured, -1 outside
  bool have_density = false;
  std::string record_path;                // JSONL record of every solve appended here (empty: off)
  size_t bytes = 0;
  std::vector<void*> allocs;

  long long vlen(int k) const { return L[k].n + (arrow ? 2 : 0); }  // allocated vector length
  long long ncg() const { return L[0].n + (arrow ? 1 : 0); }         // CG vector length

  template <typename T>
  topo_status alloc(T** ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
    if (e != cudaSuccess) return cuda_status(e, "cudaMalloc");
    allocs.push_back((void*)*ptr);
    bytes += count * sizeof(T);
    return TOPO_OK;
  }
};

namespace topo {
topo_status solver_create_internal(const topo_solver_desc* d, bool arrow, topo_solver** out);
topo_status solver_build(topo_solver* s);
topo_status solver_solve(topo_solver* s, const double* b, double* u, double tol, int use_x0,
                         topo_solve_info* info);

// Caller-stream ordering around a library call on the solver's private stream.
struct StreamGuard {
  cudaStream_t priv, user;
  cudaEvent_t in, out;
  StreamGuard(cudaStream_t priv_, cudaStream_t user_, cudaEvent_t in_, cudaEvent_t out_)
      : priv(priv_), user(user_), in(in_), out(out_) {
    cudaEventRecord(in, user);
    cudaStreamWaitEvent(priv, in, 0);
  }
  explicit StreamGuard(topo_solver* s) : StreamGuard(s->st, s->user, s->ev_in, s->ev_out) {}
  ~StreamGuard() {
    cudaEventRecord(out, priv);
    cudaStreamWaitEvent(user, out, 0);
  }
};
}  // namespace topo
