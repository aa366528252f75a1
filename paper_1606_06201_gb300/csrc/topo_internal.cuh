// Internal definitions shared by the CUDA translation units of the topology-optimisation MGCG
// library.  Grid conventions follow include/topo.h: x-fastest node and element numbering,
// interleaved DOFs, counter-clockwise local nodes (bottom face then top face in 3D).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/topo.h"
#include "pairs.cuh"

namespace topo {

constexpr int kThreads = 256;         // threads per block of the node-parallel kernels
constexpr int kRedBlocks = 4 * 152;   // blocks of the grid-stride reduction kernels (4 per SM)
constexpr int kMaxRedValues = 4;      // most values one fixed-grid reduction writes per block
constexpr int kMaxRhs = 64;

// Dimensions of one grid level.
struct Dims {
  int nx, ny, nz;  // elements per direction (nz = 1 in 2D so that products stay valid)
  int dim;
  __host__ __device__ int nnx() const { return nx + 1; }
  __host__ __device__ int nny() const { return ny + 1; }
  __host__ __device__ int nnz() const { return dim == 3 ? nz + 1 : 1; }
  __host__ __device__ long long nodes() const { return (long long)nnx() * nny() * nnz(); }
  __host__ __device__ long long dofs() const { return nodes() * dim; }
  __host__ __device__ long long elems() const { return (long long)nx * ny * (dim == 3 ? nz : 1); }
};

// Scalars of one CG recurrence, device resident (one per right-hand side).
struct CgScalars {
  double ry;       // r^T y of the current iterate
  double pq;       // p^T A p
  double rr;       // r^T r
  double ry_new;   // r~^T y~
  double ry_old;   // r~^T y (flexible beta)
  double bnorm;    // ||b||
  double alpha, beta;
  double rel;      // ||r|| / ||b||
  int iter;
  int done;        // 0 running, 1 stopped
  int status;      // topo_status
  int pad;
};

// Device-resident scalars of the interior-point method.
struct IpScalars {
  double lam, s, r;              // multiplier of the volume constraint, barrier parameters
  double V, xbar, frac;          // problem data, fraction-to-boundary factor (0.9)
  double sum_x, sum_t, res2;     // sum x, sum tilde Res3 / D, V - sum x
  double nrm_tr3, nrm_phi, nrm_psi, nrm_res1;
  double zll;                    // Z_ll = sum 1 / D
  double comp_phi, comp_psi;     // phi^T x, psi^T (xbar - x)
  double nrm_x, nrm_xu;          // ||x||, ||xbar - x||
  double alpha, dlam;            // step length, lambda direction
  int step_all;                  // 1: 0.9 rule also on phi and psi
  int pad;
};

// The SIMP model with the density filter (Sec. 9).  hat W_ij = max(0, rmin - dist(i, j)) with the
// Manhattan distance of element centres (element widths), so the stencil holds the offsets o with
// |o|_1 <= R = ceil(rmin) - 1; W = hat W diag(invS) (columns normalised, as printed).  Per-element
// buffers [m] unless noted.
constexpr int kSimpMaxR = 8;  // largest stencil half-width (rmin <= 9)
struct SimpArgs {
  double rmin = 0.0, p = 1.0;
  int R = 0;
  const double* invS = nullptr;  // 1 / (column sums of hat W)
  double* xt = nullptr;          // x~ = W x
  double* rho = nullptr;         // x~^p, the stiffness coefficients of hat K(x~)
  double* c = nullptr;           // p x~^(p-1)
  double* E = nullptr;           // u_e^T K0 u_e
  double* e3 = nullptr;          // 1/2 W^T (c E), the energy term of the modified row 3
  double* gh = nullptr;          // [m * ne] c_e g_e, the element columns of hat B = G diag(c) W
  double* th = nullptr;          // W (tilde Res3 / D)
  double* Dm = nullptr;          // W D^{-1} e, the row sums of W D^{-1} W^T: the hierarchy's weights
  double* ea = nullptr;          // scratch
  double* eb = nullptr;          // scratch
};

// Device-resident scalars of the OC bisection.
struct OcScalars {
  double lo, hi, tau, lam_last;
  double V, xlow, xbar;
  int steps, pad;
};

// Per-level data of the multigrid hierarchy.  Level 0 is the finest.
struct Level {
  Dims d;
  long long n = 0, m = 0;          // DOFs, elements
  uint8_t* fixed = nullptr;        // [n] 1 = fixed DOF
  double* Ae = nullptr;            // coarse levels: element matrices, entry-major [ne*ne][m] FP64
  float* Ae32 = nullptr;           // FP32 copy (mixed precision)
  void* Aem = nullptr;             // the V-cycle's element matrices element-major, kAemStride
                                   // entries per element (levels of the single-block deep tail)
  double* invd = nullptr;          // 1 / diag(A) [n] (1 on fixed DOFs)
  float* invd32 = nullptr;
  double* omega_dev = nullptr;     // per-level Jacobi damping (adaptive damping only)
  double* lam_dev = nullptr;       // lambda_max(D^{-1} A) estimate (Chebyshev smoother)
  void* cd = nullptr;              // Chebyshev direction vector
  double* w = nullptr;             // arrow column Z_ul on this level (IP systems) [n]
  float* w32 = nullptr;
  void* b = nullptr;               // V-cycle right-hand side   [nrhs][n] (FP64 or FP32)
  void* z = nullptr;               // V-cycle iterate
  void* t = nullptr;               // ping-pong / residual scratch
};

// Coefficients of the 2D Q1 element matrix in its butterfly basis (kernels_q1.cu):
// K0 = T^T Khat T with Khat built from c11, c12, c22 (normal block), c33 (shear), cH, cHp
// (hourglass); kd = K0_ii (all diagonal entries are equal for the square element).
struct Q1Coef {
  double c11, c12, c22, c33, cH, cHp, kd;
};

// Coefficients of the 3D hex K0 in the element's Walsh-Hadamard basis (kernels_hex.cu): normal
// block a (diagonal) and b, shear s, bilinear pairs p and q, the triple d and e, trilinear h.
struct HexCoef {
  double a, b, s, p, q, d, e, h;
};

// Host-side error reporting.
void set_error(const std::string& msg);
topo_status cuda_status(cudaError_t e, const char* what);

#define TOPO_CUDA(call)                                         \
  do {                                                          \
    cudaError_t _e = (call);                                    \
    if (_e != cudaSuccess) return topo::cuda_status(_e, #call); \
  } while (0)

#define TOPO_CHECK_LAUNCH(what)                                 \
  do {                                                          \
    cudaError_t _e = cudaGetLastError();                        \
    if (_e != cudaSuccess) return topo::cuda_status(_e, what);  \
  } while (0)

// ---- Index checks of the debug build --------------------------------------------------------
// Built with -DTOPO_BOUNDS_CHECK, the operator kernels check the indices they compute against the
// sizes of the buffers they address.  An index outside [0, size) is never used: a checked load
// reads entry 0 instead (TOPO_IDX) and a checked store is skipped (TOPO_IN); the first such index
// of each translation unit is recorded with its source line, and every solve then returns
// TOPO_E_BOUNDS (topo_bounds_report reads the records).  Nothing traps.  Without the macro both
// checks are constants and cost nothing.
struct BoundsRecord {
  unsigned long long count;  // indices found outside their range since the last reset
  long long index, size;     // the first of them and the size it was checked against
  int line, pad;             // its source line
};
using BoundsReader = cudaError_t (*)(BoundsRecord* out, bool reset);
// Registers the record reader of one translation unit (host, at load time); returns its number.
int register_bounds_reader(BoundsReader reader, const char* file);

#ifdef TOPO_BOUNDS_CHECK
static __device__ BoundsRecord g_topo_bounds;  // (one per translation unit)
__device__ __noinline__ static bool topo_out_of_bounds(long long i, long long n, int line) {
  if (atomicAdd(&g_topo_bounds.count, 1ull) == 0ull) {
    g_topo_bounds.index = i;
    g_topo_bounds.size = n;
    g_topo_bounds.line = line;
  }
  return false;
}
#define TOPO_IN(i, n)                                                              \
  ((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n) ||      \
   topo::topo_out_of_bounds((long long)(i), (long long)(n), __LINE__))
#define TOPO_IDX(i, n) (TOPO_IN(i, n) ? (i) : 0)
static cudaError_t read_bounds_record(BoundsRecord* out, bool reset) {
  cudaError_t e = cudaMemcpyFromSymbol(out, g_topo_bounds, sizeof(BoundsRecord));
  if (e == cudaSuccess && reset) {
    const BoundsRecord zero = {};
    e = cudaMemcpyToSymbol(g_topo_bounds, &zero, sizeof(BoundsRecord));
  }
  return e;
}
[[maybe_unused]] static const int g_bounds_reader_id = register_bounds_reader(&read_bounds_record, __FILE__);
#else
#define TOPO_IN(i, n) ((void)(n), true)
#define TOPO_IDX(i, n) ((void)(n), (i))
#endif

// A named NVTX range for the duration of a scope: the phases of the method (hierarchy build, MGCG
// solve, IP Newton step, OC step) show up as ranges in profilers (ncu --nvtx, Nsight Systems); with
// no tool attached a push or pop costs a few nanoseconds.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Programmatic dependent launch (optional, TOPO_PDL=1): every kernel waits for its stream
// predecessor's completion before touching memory (griddepcontrol.wait) and at once lets its own
// successor start launching.  Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_prologue() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

bool pdl_enabled();

template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                   Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Node coordinates from a linear node index with 32-bit division (grids hold < 2^31 nodes; the
// solver checks this at creation): i fastest, then j, then k.
__device__ __forceinline__ void node_coords(long long node, int nnx, int nny, int dim, int& i,
                                            int& j, int& k) {
  const unsigned nd = (unsigned)node;
  const unsigned q = nd / (unsigned)nnx;
  i = (int)(nd - q * (unsigned)nnx);
  if (dim == 3) {
    const unsigned r = q / (unsigned)nny;
    j = (int)(q - r * (unsigned)nny);
    k = (int)r;
  } else {
    j = (int)q;
    k = 0;
  }
}

// Rounded products that the compiler may not contract into a later addition: the fused V-cycle
// kernels form values that the unfused ones store to memory, and must round them the same way.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Output of one DOF row of the node-parallel operator kernels: mode 1 b - A v; modes 2 and 4 one
// Jacobi sweep v + omega invd (b - A v); mode 3 the first sweep from zero omega invd b.  The
// roundings are spelled out (no contraction left to the compiler), so that every kernel that
// forms these rows gives the same bits.
template <int MODE, typename T>
__device__ __forceinline__ T node_out(T acc, T v, T b, T invd, T omega) {
  if constexpr (MODE == 1) return b - acc;
  else if constexpr (MODE == 2 || MODE == 4) return fma(mul_rn(omega, invd), b - acc, v);
  else if constexpr (MODE == 3) return mul_rn(mul_rn(omega, invd), b);
  else return acc;
}

// z_row = sum_k Ainv[row][k] b[k] by one warp: lane-strided FP64 sums, then a butterfly
// (COH: b read from L2, for data written earlier in the same launch by other blocks).
template <bool COH, typename T>
__device__ __forceinline__ double dense_row_dot(int n, const double* __restrict__ row, const T* b,
                                                int lane) {
  double s = 0.0;
  for (int k = lane; k < n; k += 32) {
    T bk;
    if constexpr (COH) bk = __ldcg(b + k);
    else bk = b[k];
    s = fma(row[k], double_of(bk), s);  // (integer widening: no FP64 conversion instruction)
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// The same product for an FP32 V-cycle with Ainv held as float pairs hi + lo (split once per
// build): pair products and sums on the FP32 pipe (about 48 bits), z rounded to FP32.  The FP64
// pipe of this part issues two lane operations per clock per SM, so the FP64 form of a 90-row
// coarsest solve (8,100 multiply-adds and 14,400 butterfly adds) took 8-9 us in one block.
__device__ __forceinline__ f2 df_fma_f(f2 a, float b, f2 c) {  // a b + c, b a float
  const float p = __fmul_rn(a.h, b);
  float e = __fmaf_rn(a.h, b, -p);
  e = __fmaf_rn(a.l, b, e);
  return df_add(fast_two_sum(p, e), c);
}
template <bool COH>
__device__ __forceinline__ f2 dense_row_dot_df(int n, const float2* __restrict__ row,
                                               const float* b, int lane) {
  f2 s = {0.0f, 0.0f};
  for (int k = lane; k < n; k += 32) {
    float bk;
    if constexpr (COH) bk = __ldcg(b + k);
    else bk = b[k];
    const float2 a = row[k];
    s = df_fma_f(f2{a.x, a.y}, bk, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    s = df_add(s, f2{__shfl_xor_sync(0xffffffffu, s.h, o), __shfl_xor_sync(0xffffffffu, s.l, o)});
  return s;
}

// Deep levels of the 2D V-cycle fused into one launch (kernels_fe.cu): levels tail_from ..
// coarsest, run by one thread-block cluster per right-hand side.
#ifndef TOPO_TAIL_CLUSTER
#define TOPO_TAIL_CLUSTER 8
#endif
#ifndef TOPO_TAIL_THREADS
#define TOPO_TAIL_THREADS 256
#endif
// Measured on the 2048 x 1024 solve (9 levels, ms per hierarchy build + solve): unfused 7.95;
// fused from the level of 2145 nodes 7.93-8.02, from 8385 nodes 8.18-8.28, from 561 nodes 7.92.
// Graph launches of the small kernels cost about as much as the L2 round trips of a fused phase,
// so the fused part starts where a level fits in one pass of the cluster's threads.
#ifndef TOPO_TAIL_NODES
#define TOPO_TAIL_NODES 1024
#endif
constexpr int kTailMax = 8;                      // levels in the fused part, coarsest included
constexpr int kTailCluster = TOPO_TAIL_CLUSTER;  // blocks per cluster (above 8: non-portable)
constexpr int kTailThreads = TOPO_TAIL_THREADS;
constexpr long long kTailNodes = TOPO_TAIL_NODES;  // most nodes of the first fused level

template <typename T>
struct TailArgs {
  int nl;        // fused levels, the last one the coarsest
  int nu1, nu2;
  int nc;        // coarsest DOFs (Ainv is nc x nc)
  T omega;
  const double* Ainv;
  const float2* AinvDF;  // Ainv as float pairs (FP32 V-cycles)
  Dims d[kTailMax];
  const T* Ae[kTailMax];
  const T* Aem[kTailMax];  // element-major copies (single-block form)
  const T* invd[kTailMax];
  const uint8_t* fixed[kTailMax];
  T* b[kTailMax];  // b[0]: the restricted residual from the level above
  T* z[kTailMax];
  T* t[kTailMax];
  // single-block form (k_vcycle_tail1): byte offsets of each level's element matrices, vectors
  // and mask in shared memory, and the bytes in all
  unsigned off_m[kTailMax], off_z[kTailMax], off_t[kTailMax], off_b[kTailMax], off_d[kTailMax],
      off_f[kTailMax];
  unsigned off_bar;  // the mbarrier of the bulk copies
  unsigned smem;
  unsigned long long wait_ns;  // bound of the first wait for the bulk copies (0: expire at once)
};
// Threads of the single-block deep tail (FP32; FP64 takes half): 1024 measured faster than 512
// once the node rows fit in 64 registers (see the kernel).
#ifndef TOPO_TAIL1_THREADS
#define TOPO_TAIL1_THREADS 1024
#endif
constexpr int kTail1Threads = TOPO_TAIL1_THREADS;
// Entries per element of the element-major copies of the deep levels' 8 x 8 matrices: 64 padded
// to 68, so that 16-byte loads of consecutive elements fall in distinct shared-memory banks.
constexpr int kAemStride = 68;
template <typename T>
cudaError_t launch_pack_element_major(long long m, const T* Ae, T* Aem, cudaStream_t st);

inline unsigned blocks_for(long long n, int threads = kThreads) {
  return (unsigned)((n + threads - 1) / threads);
}

// ---- kernels (launchers), defined in kernels_*.cu --------------------------------------------
// Element stiffness on the host (2-point Gauss per direction).
void element_stiffness_host(int dim, double E, double nu, double* K0);

// Operator application on one level.  mode: 0 y = A v; 1 y = b - A v; 2 y = v + omega invd (b - A v);
// 3 y = omega invd b (first Jacobi sweep from zero, v unused); 2D stored element matrices only:
// 4 = mode 2 on v = omega invd b (the first two sweeps from zero, v unused).
// x != nullptr: finest level with element matrices x_e K0; otherwise Ae holds element matrices.
// nrhs vectors of length n.
// w != nullptr adds the arrow column: y_u += w v_lambda with v_lambda = v[n] (nrhs = 1).
template <typename T>
cudaError_t launch_apply(const Dims& d, int mode, const T* K0, const T* x, const T* Ae, const T* v,
                         const T* b,
                         T* y, const T* invd, T omega, const uint8_t* fixed, int nrhs,
                         const CgScalars* sc, cudaStream_t st, const T* w = nullptr);
// Fused deep part of the V-cycle (Jacobi smoothing, element matrices on every fused level but
// the coarsest): the result of the first fused level ends in z[0] or t[0] as in the unfused
// cycle (tail_result).
template <typename T>
cudaError_t launch_vcycle_tail(const TailArgs<T>& a, int nrhs, const CgScalars* sc,
                               cudaStream_t st);
cudaError_t prepare_tail_kernels();
// The same levels in the shared memory of one block per right-hand side (no cluster barrier, no
// L2 round trip between phases).  tail1_layout fills a.off_* and a.smem and returns whether they
// fit in a block's shared memory; launch_vcycle_tail1 leaves the first level's result in z[0].
template <typename T>
bool tail1_layout(TailArgs<T>& a);
template <typename T>
cudaError_t launch_vcycle_tail1(const TailArgs<T>& a, int nrhs, const CgScalars* sc,
                                cudaStream_t st);
// First coarse level of a 2D grid, matrix-free from the finest densities xf and the four child
// matrices C (same modes as launch_apply).
template <typename T>
cudaError_t launch_apply_l1(const Dims& d, int mode, const T* C, const T* xf, const T* v,
                            const T* b, T* y, const T* invd, T omega, const uint8_t* fixed,
                            int nrhs, const CgScalars* sc, cudaStream_t st);
// y = A v in FP64 on the finest level with a fused per-block partial of v^T y (for p^T A p).
cudaError_t launch_apply_dot_fine(const Dims& d, const double* K0, const double* x, const double* v,
                                  double* y,
                                  const uint8_t* fixed, int nrhs, double* partials,
                                  unsigned* counters, CgScalars* sc, cudaStream_t st);
// arrow: the trailing lambda entry is carried by the identity (restriction copies it,
// prolongation adds it).
template <typename T>
cudaError_t launch_restrict(const Dims& fine, const T* rf, T* rc, const uint8_t* fixed_c, int nrhs,
                            const CgScalars* sc, cudaStream_t st, int arrow = 0);
template <typename T>
cudaError_t launch_prolong_add(const Dims& fine, const T* zc, T* zf, const uint8_t* fixed_f,
                               int nrhs, const CgScalars* sc, cudaStream_t st, int arrow = 0);
// 2D level with stored element matrices Ae (no arrow): y = v + omega invd (b - A v) with
// v = z + P zc (prolongation and correction, then the first post-smoothing sweep) in one launch,
// with the bits of launch_prolong_add followed by launch_apply mode 2.
// Levels at or below this many nodes take launch_apply2_prolong: on the 2048 x 1024 hierarchy
// levels 3-5 gain 0.3-1.8 us each; on level 2 (132k nodes) the parity classes' strided accesses
// made it 4 us slower than the two kernels.
constexpr long long kApply2ProlongNodes = 65536;
template <typename T>
cudaError_t launch_apply2_prolong(const Dims& d, const T* Ae, const T* z, const T* zc, const T* b,
                                  T* y, const T* invd, T omega, const uint8_t* fixed, int nrhs,
                                  const CgScalars* sc, cudaStream_t st);
cudaError_t launch_inv_diag(const Dims& d, const double* K0, const double* x, const double* Ae,
                            const uint8_t* fixed, double* invd, cudaStream_t st);
// FP32 inverse diagonal of a coarse level from its FP32 element matrices.
cudaError_t launch_inv_diag32(const Dims& d, const float* Ae, const uint8_t* fixed, float* invd,
                              cudaStream_t st);
cudaError_t launch_element_energy(const Dims& d, const double* K0, const double* u,
                                  const double* lam, double* out, double scale, cudaStream_t st);

// Finest-level 2D Q1 operator, warp-sweep kernels (kernels_q1.cu); same modes as launch_apply.
// b_c = P^T (b - K(x) v) on the finest level in one pass (the residual is not stored): the same
// bits as launch_q1_apply mode 1 followed by launch_restrict.  bc, fixed_c: the first coarse
// level's right-hand sides [nrhs][n_c] and mask.
template <typename T>
cudaError_t launch_q1_resrestrict(int nx, int ny, const Q1Coef& coef, const T* x, const T* v,
                                  const T* b, T* bc, const uint8_t* fixed,
                                  const uint8_t* fixed_c, int nrhs, const CgScalars* sc,
                                  cudaStream_t st);
template <typename T>
cudaError_t launch_q1_apply(int nx, int ny, int mode, const Q1Coef& coef, const T* x, const T* v,
                            const T* b, T* y, T omega, const uint8_t* fixed, int nrhs,
                            const CgScalars* sc, cudaStream_t st);
cudaError_t launch_q1_apply_dot(int nx, int ny, const Q1Coef& coef, const double* x,
                                const double* v, double* y, const uint8_t* fixed, int nrhs,
                                double* partials, unsigned* counters, CgScalars* sc,
                                cudaStream_t st);
long long q1_partial_blocks(int nx, int ny);
// The FP32 finest-level sweeps with two node columns per lane (kernels_q1w.cu): the same outputs
// as launch_q1_apply, launch_q1_fused, launch_q1_resrestrict and launch_q1_smooth_beta for T =
// float (the fused dot of the last one summed in another order).  rows: the strip height of the
// fine sweeps (0: about one wave of warps; the residual-restriction takes rows / 2 coarse rows).
// fixed: the finest mask as node pairs with an even row stride ((nx + 2) / 2 words per node row,
// the pad node zero; topo_solver::fixed_pad).
cudaError_t launch_q1w_apply(int nx, int ny, int mode, const Q1Coef& coef, const float* x,
                             const float* v, const float* b, float* y, float omega,
                             const unsigned* fixed, int nrhs, const CgScalars* sc, cudaStream_t st,
                             int rows = 0);
cudaError_t launch_q1w_fused(int nx, int ny, int mode, const Q1Coef& coef, const float* x,
                             const float* t, const float* zc, const float* b, float* y,
                             float omega, const unsigned* fixed, int nrhs, const CgScalars* sc,
                             cudaStream_t st, int rows = 0);
cudaError_t launch_q1w_smooth_beta(int nx, int ny, const Q1Coef& coef, const float* x,
                                   const float* v, const float* b, float* y, float omega,
                                   const unsigned* fixed, int nrhs, const double* r,
                                   double* partials, unsigned* counters, CgScalars* sc,
                                   cudaStream_t st, int rows = 0);
cudaError_t launch_q1w_resrestrict(int nx, int ny, const Q1Coef& coef, const float* x,
                                   const float* v, const float* b, float* bc,
                                   const unsigned* fixed, const uint8_t* fixed_c, int nrhs,
                                   const CgScalars* sc, cudaStream_t st, int rows = 0);
long long q1w_partial_blocks(int nx, int ny);
// 3D finest-level outer operator in the Walsh-Hadamard basis (kernels_hex.cu): element forces into
// R (24 x elems per right-hand side), then a node gather with p^T q and alpha.  hex_coefficients
// returns false when T^T Khat T does not reproduce K0 (the generic kernel is then used).
bool hex_coefficients(const double* K0, HexCoef& c);
cudaError_t launch_hex_apply_dot(const Dims& d, const HexCoef& c, const double* x, const double* v,
                                 double* y, const uint8_t* fixed, int nrhs, double* R,
                                 double* partials, unsigned* counters, CgScalars* sc,
                                 cudaStream_t st);
// The same in pair-of-FP32 arithmetic (about 48 bits; xdf: the densities as float pairs).
cudaError_t launch_hex_apply_dot_df(const Dims& d, const HexCoef& c, const float2* xdf,
                                    const double* v, double* y, const uint8_t* fixed, int nrhs,
                                    double* R, double* partials, unsigned* counters, CgScalars* sc,
                                    cudaStream_t st);
// The same operators in the tile form (kernels_hex.cu): element forces through shared memory, one
// launch, no force buffer; q has the bits of the buffered form.  x: FP64 densities, or float pairs
// when `pairs`.
// Counts the inputs where the integer FP64 <-> FP32 conversions differ from the hardware ones.
cudaError_t launch_check_conversions(const double* d, const float* f, long long n,
                                     unsigned long long* bad, cudaStream_t st);
template <typename T>
cudaError_t launch_hex_tile_sweep_beta(const Dims& d, int form, const HexCoef& c, const T* K0,
                                       const T* x, const T* v, const T* b, T* y, const T* invd,
                                       T omega, const uint8_t* fixed, int nrhs, CgScalars* sc,
                                       const double* rdot, double* partials, unsigned* counters,
                                       cudaStream_t st);
cudaError_t prepare_hex_tile_kernels();
cudaError_t launch_hex_tile_apply_dot(const Dims& d, const HexCoef& c, const void* x, bool pairs,
                                      const double* v, double* y, const uint8_t* fixed, int nrhs,
                                      double* partials, unsigned* counters, CgScalars* sc,
                                      cudaStream_t st);
// Finest-level 3D V-cycle operator (modes 0-2 of launch_apply) in the tile form: form 0 in the
// Walsh-Hadamard basis, 1 with the element rows of K0 (the bits of the node-parallel kernel), 2 the
// same product on the tensor cores (3 x TF32, FP32 vectors only).
template <typename T>
cudaError_t launch_hex_tile_sweep(const Dims& d, int mode, int form, const HexCoef& c,
                                  const T* K0, const T* x, const T* v, const T* b, T* y,
                                  const T* invd, T omega, const uint8_t* fixed, int nrhs,
                                  const CgScalars* sc, cudaStream_t st);
// Fused pairs of finest-level V-cycle steps (same bits as the separate steps): mode 4 = the first
// two Jacobi sweeps from zero (b -> y); mode 5 = prolongation and correction t + P zc followed by
// one Jacobi sweep (t, zc -> y).  zc: the first coarse level's vector.
template <typename T>
cudaError_t launch_q1_fused(int nx, int ny, int mode, const Q1Coef& coef, const T* x, const T* t,
                            const T* zc, const T* b, T* y, T omega, const uint8_t* fixed,
                            int nrhs, const CgScalars* sc, cudaStream_t st);
// The same q = K(x) p with p^T q and alpha in pair-of-FP32 arithmetic (about 48 bits), with the
// densities split once per hierarchy build (launch_split_df).
cudaError_t launch_q1_apply_dot_df(int nx, int ny, const Q1Coef& coef, const float2* xdf,
                                   const double* v, double* y, const uint8_t* fixed, int nrhs,
                                   double* partials, unsigned* counters, CgScalars* sc,
                                   cudaStream_t st);
cudaError_t launch_split_df(const double* x, float2* out, long long m, cudaStream_t st);
// flag = 1 if some x_i is not finite and > 0 (flag zeroed by the caller); x32 = (float) x and
// xdf = x as float pairs where not null.
cudaError_t launch_prepare_x(const double* x, long long m, int* flag, float* x32, float2* xdf,
                             cudaStream_t st);
// Jacobi sweep (mode 2) on the 2D finest level fused with r^T y against the FP64 CG residual r and
// the beta of Algorithm PCG (last smoothing sweep of the preconditioner).
template <typename T>
cudaError_t launch_q1_smooth_beta(int nx, int ny, const Q1Coef& coef, const T* x, const T* v,
                                  const T* b, T* y, T omega, const uint8_t* fixed, int nrhs,
                                  const double* r, double* partials, unsigned* counters,
                                  CgScalars* sc, cudaStream_t st);
// 2D level with stored (entry-major) element matrices, warp-sweep data movement; w: arrow column.
template <typename T>
cudaError_t launch_ae_sweep(int nx, int ny, int mode, const T* Ae, const T* v, const T* b, T* y,
                            T omega, const T* invd, const uint8_t* fixed, const T* w, int nrhs,
                            const CgScalars* sc, cudaStream_t st);
// First coarse level of the 2D Q1 hierarchy, matrix-free in FP32 (P^T K(x) P element by element);
// nx, ny = coarse elements, xf = finest densities.
// mode 4, 5: the fused pairs of steps of launch_q1_fused on this level (zc: the next coarser
// level's vector for mode 5).
cudaError_t launch_q1g_apply(int nx, int ny, int mode, const Q1Coef& coef, const float* xf,
                             const float* v, const float* b, float* y, float omega,
                             const float* invd, const uint8_t* fixed, int nrhs,
                             const CgScalars* sc, cudaStream_t st, const float* zc = nullptr);

// Hierarchy construction (kernels_rap.cu).
// g, Dinv != nullptr: add the rank-one terms (P_c^T g_c)(P_c^T g_c)^T Dinv_c of Z.
// T = double or float (arithmetic and storage); the rank-one terms g, Dinv need T = double.
// Ch / C2h [host, FP64]: the same tables as C / C2; given in 2D, one thread per coarse element
// takes them as kernel parameters (the same bits as the entry-parallel kernels).
template <typename T>
cudaError_t launch_rap_from_fine(const Dims& fine, const T* C, const T* x, T* Ac, cudaStream_t st,
                                 const double* g = nullptr, const double* Dinv = nullptr,
                                 const double* Ch = nullptr);
// TI: stored type of the finer level's matrices; TO: arithmetic and stored type of the result
// (double/double, float/float, float/double).
template <typename TI, typename TO>
cudaError_t launch_rap_coarse(const Dims& fine, const TI* Af, TO* Ac, cudaStream_t st);
// Second coarse level from the finest densities with the 4^dim composite matrices C2.
template <typename T>
cudaError_t launch_rap2_from_fine(const Dims& fine, const T* C2, const T* x, T* Ac,
                                  cudaStream_t st, const double* C2h = nullptr);
// Inverse diagonal of the first coarse level from the finest densities and the child matrices.
template <typename T>
cudaError_t launch_inv_diag_l1(const Dims& coarse1, const T* C, const T* xf,
                               const uint8_t* fixed, T* invd, cudaStream_t st);
// Dense operator of a level with leading dimension ld; with an arrow (w != nullptr) the row and
// column n hold w (zero on fixed DOFs) and A[n][n] = *zll.  g, Dinv: rank-one terms (finest level).
cudaError_t launch_assemble_dense(const Dims& d, const double* K0, const double* x,
                                  const double* Ae,
                                  const uint8_t* fixed, double* A, cudaStream_t st,
                                  long long ld = 0, const double* w = nullptr,
                                  const double* zll = nullptr, const double* g = nullptr,
                                  const double* Dinv = nullptr);
// Ainv = A^{-1} for the dense SPD coarsest matrix; info[0] = 0 or k+1 (pivot k failed).  With
// allow_ns and n small enough: FP32 Gauss-Jordan + FP64 Newton-Schulz in scratch
// (coarse_scratch_doubles(n) doubles), *ns_bad set if that did not reach FP64 accuracy, in which
// case the Cholesky kernels (always enqueued) recompute it; otherwise Cholesky (with the pivot
// floor) + triangular inverse.
cudaError_t launch_cholesky_inverse(int n, double* A, double* Ainv, int* info, cudaStream_t st,
                                    double* scratch = nullptr, int* ns_bad = nullptr,
                                    bool allow_ns = false);
size_t coarse_scratch_doubles(int n);
// Shared-memory limits of the coarsest-level kernels (call once, outside stream capture).
cudaError_t prepare_coarse_kernels(int n);
template <typename T>
cudaError_t launch_dense_solve(int n, const double* Ainv, const float2* AinvDF, const T* b, T* z,
                               int nrhs,
                               const CgScalars* sc, cudaStream_t st);
cudaError_t launch_convert_d2f(const double* a, float* b, long long n, cudaStream_t st);
cudaError_t launch_convert_f2d(const float* a, double* b, long long n, cudaStream_t st);
cudaError_t launch_check_positive(const double* x, long long m, int* flag, cudaStream_t st);

// CG vector kernels (kernels_pcg.cu).
// z = 0, r = -b (b masked on the fixed DOFs below n_mask), rv = (TV) r (rv may be null) and the
// start scalars, in one pass over the caller's b.
template <typename TV>
cudaError_t launch_cg_init_zero(long long n, long long n_mask, int nrhs, const double* b,
                                const uint8_t* fixed, double* z, double* r, TV* rv,
                                double* partials, unsigned* counters, CgScalars* sc, double tol,
                                int max_iter, cudaStream_t st);
// z += alpha p per right-hand side with alpha != 0: the iterate update of the iteration that
// ended the solve (k_cg_p applies it otherwise).
cudaError_t launch_cg_finish_z(long long n, int nrhs, const double* p, double* z,
                               const CgScalars* sc, cudaStream_t st);
cudaError_t launch_cg_init(long long n, int nrhs, const double* b, double* z, double* r,
                           const double* Az, int use_x0, double* partials, unsigned* counters,
                           CgScalars* sc, double tol, int max_iter, cudaStream_t st);
template <typename TV>
cudaError_t launch_cg_start_p(long long n, int nrhs, const double* r, const TV* y, double* p,
                              TV* y_old, int flexible, double* partials, unsigned* counters,
                              CgScalars* sc, cudaStream_t st);
template <typename TV>
cudaError_t launch_cg_update(long long n, int nrhs, double* z, double* r, const double* p,
                             const double* q, TV* rv, double* partials, unsigned* counters,
                             CgScalars* sc, double tol, int max_iter, cudaStream_t st);
template <typename TV>
cudaError_t launch_cg_direction(long long n, int nrhs, const double* r, const TV* y, double* p,
                                TV* y_old, int flexible, double* partials, unsigned* counters,
                                CgScalars* sc, cudaStream_t st, double* z);
// p = -y + beta p (beta already in the scalars), y_old = y if flexible.
template <typename TV>
cudaError_t launch_cg_p(long long n, int nrhs, const TV* y, double* p, TV* y_old, int flexible,
                        CgScalars* sc, cudaStream_t st, double* z);
cudaError_t launch_dot(long long n, int nrhs, const double* a, const double* b, double* partials,
                       unsigned* counters, double* out, cudaStream_t st);
// Power iteration for lambda_max(D^{-1} A): v <- D^{-1} A v / ||.||_D (y = A v supplied by the
// caller); est[0] = Rayleigh quotient, est[1] = normalisation.  finish: omega_k = min(omega,
// c / (1.05 est[0])) written to omega_dev and folded into invd (invd <- omega_k invd).
cudaError_t launch_power_init(long long n, int arrow, double* v, const uint8_t* fixed,
                              cudaStream_t st);
cudaError_t launch_power_step(long long n, int arrow, const double* v, const double* y,
                              const double* invd, const double* zll, double* w, double* partials,
                              unsigned* counters, double* est, cudaStream_t st);
cudaError_t launch_power_finish(long long n, const double* est, double omega, double c,
                                double* omega_dev, double* invd, cudaStream_t st);
// lam_dev <- est[0] (the Chebyshev smoother keeps the estimate instead of folding it into invd).
cudaError_t launch_power_store(const double* est, double* lam_dev, cudaStream_t st);
// One Chebyshev smoothing step (see kernels_pcg.cu): t = b - A z (t = b for step 0 from z = 0,
// z_zero = 1, which overwrites z).
template <typename T>
cudaError_t launch_cheb_update(long long n, int nrhs, int step, int z_zero, const double* lam_dev,
                               double alpha, const T* invd, const T* t, T* d, T* z,
                               const uint8_t* fixed, const CgScalars* sc, cudaStream_t st);
// Sets the while-loop condition of the persistent CG graph (1 while any right-hand side runs).
cudaError_t launch_loop_cond(cudaGraphConditionalHandle handle, const CgScalars* sc, int nrhs,
                             int max_iter, cudaStream_t st);
cudaError_t launch_mask_copy(long long n, long long n_mask, int nrhs, const double* src,
                             double* dst, const uint8_t* fixed, cudaStream_t st);
// p^T q and alpha = r^T y / p^T q (breakdown checks as in the fused operator kernel).
cudaError_t launch_cg_alpha(long long n, int nrhs, const double* p, const double* q,
                            double* partials, unsigned* counters, CgScalars* sc, cudaStream_t st);

// IP and OC kernels (kernels_ip.cu).
// wdev != nullptr: the damping of the lambda entry is read from the device (the u-part then
// takes omega folded into invd, with omega = 1 passed here).
template <typename T>
cudaError_t launch_z_apply_fine(const Dims& d, int mode, const T* K0, const T* x, const T* g,
                                const T* Dinv, T* se, const T* v, const T* b, T* y, const T* invd,
                                T omega, const uint8_t* fixed, const double* zll, double* partials,
                                unsigned* counter, const CgScalars* sc, cudaStream_t st,
                                const double* wdev = nullptr);
// Coarse level of an IP system in one launch: node rows with the arrow column w, and the lambda
// row w^T v_u + Z_ll v_lambda from a fixed-grid reduction in the same kernel (y[n] per mode, with
// omega_l or *wdev for the lambda entry).  Modes 0-3 as launch_apply; mode 4 (2D only) the first
// two sweeps from zero.  nrhs = 1.
template <typename T>
cudaError_t launch_apply_arrow(const Dims& d, int mode, const T* Ae, const T* v, const T* b, T* y,
                               const T* invd, T omega, const uint8_t* fixed, const T* w,
                               const double* zll, double omega_l, const double* wdev,
                               double* partials, unsigned* counter, const CgScalars* sc,
                               cudaStream_t st);
// sa != nullptr: the SIMP residuals (Sec. 9): x~, rho, c from x; F3 with the filtered energy
// term; rhs, w, invd of Z with hat B = G diag(c) W, whose element-local hierarchy takes the
// row sums of W D^{-1} W^T (sa->Dm) as weights and the columns sa->gh.  Dinv keeps the exact 1/D.
cudaError_t launch_ip_residuals(const Dims& d, const double* K0, const double* u, const double* x,
                                const double* phi, const double* psi, const double* f,
                                const uint8_t* fixed, IpScalars* ip, double* g, double* tR3,
                                double* Dinv, double* t, double* rhs, double* w, double* invd,
                                double* partials, unsigned* counter, cudaStream_t st,
                                const SimpArgs* sa = nullptr);
cudaError_t launch_ip_recover_update(const Dims& d, const double* g, const double* du,
                                     const double* tR3, const double* Dinv, double* u, double* x,
                                     double* phi, double* psi, double* dx, double* dphi,
                                     double* dpsi, IpScalars* ip, double* partials,
                                     unsigned* counter, cudaStream_t st,
                                     const SimpArgs* sa = nullptr);
// 1 / column sums of hat W (SIMP filter).
cudaError_t launch_filter_colsum(const Dims& d, double rmin, int R, double* invS, cudaStream_t st);
// x~ = W x, rho = x~^p, c = p x~^(p-1).
cudaError_t launch_simp_density(const Dims& d, const SimpArgs& sa, const double* x,
                                cudaStream_t st);
// The exact SIMP augmented operator y = Z v (MODE 0):  a_e = gh_e^T v_e;
// sb = Dinv (W^T a + v_lambda), y_lambda = sum sb;  se = W sb;  y_u = hat K v + sum_e gh_e se_e
// (the node pass in float pairs when df).
cudaError_t launch_simp_z_apply(const Dims& d, const double* K0, const double* rho,
                                const double* gh, const double* Dinv, const double* invS,
                                double rmin, int R, double* ea, double* eb, double* se,
                                const double* v, double* y, const uint8_t* fixed,
                                double* partials, unsigned* counter, const CgScalars* sc,
                                cudaStream_t st, bool df);
// The finest-level Z operator y = Z v (MODE 0) of mixed-precision IP systems: the element pass in
// FP64 (s_e and the lambda row), the node pass in float pairs (about 48 bits).
cudaError_t launch_z_apply_fine_df(const Dims& d, const double* K0, const double* x,
                                   const double* g, const double* Dinv, double* se,
                                   const double* v, double* y, const uint8_t* fixed,
                                   const double* zll, double* partials, unsigned* counter,
                                   const CgScalars* sc, cudaStream_t st);
cudaError_t launch_oc_bisection(long long m, const double* x, const double* E, OcScalars* oc,
                                int steps, double* xout, double* partials, unsigned* counter,
                                cudaStream_t st);
cudaError_t launch_average(long long m, const double* a, const double* b, double* out,
                           cudaStream_t st);
cudaError_t launch_pow_inplace(long long m, double* E, double q, cudaStream_t st);

}  // namespace topo
