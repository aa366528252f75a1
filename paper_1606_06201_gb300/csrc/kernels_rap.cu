// Hierarchy construction: Galerkin coarse operators A_{k-1} = P^T A_k P (Sec. 5.1) computed
// element by element, the dense coarsest operator, its Cholesky factorisation and inverse (the
// exact coarsest-grid solve of Algorithm MG), and the application of that inverse.
//
// Element-local Galerkin product: the bilinear (trilinear) prolongation of Sec. 7 interpolates
// the values inside a coarse element from that element's own nodes only, so restricted to one
// fine child element c of coarse element E it is a small matrix P_c (node weights W_c times the
// identity on components) and  P^T A P = sum_E L_E^T ( sum_{c in E} P_c^T A_c P_c ) L_E.
// For the first coarsening A_c = x_c K0, so sum_c x_c (P_c^T K0 P_c) with four (eight) constant
// matrices C_c = P_c^T K0 P_c prepared on the host.
#include <type_traits>

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

// 1-D weight of the coarse-element-local node coordinate q in {0,1} at the fine position
// p in {0,1,2} (in fine units, inside the coarse element): 1 - |p - 2q| / 2.
__device__ __forceinline__ double w1(int p, int q) {
  const int dd = p - 2 * q;
  return dd == 0 ? 1.0 : ((dd == 1 || dd == -1) ? 0.5 : 0.0);
}

// W_c[a][A]: weight of coarse local node A at fine local node a of child c.
template <int DIM>
__device__ __forceinline__ double wchild(int c, int a, int A) {
  const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
  double w = w1(cx + loc_ox(a), loc_ox(A)) * w1(cy + loc_oy(a), loc_oy(A));
  if (DIM == 3) w *= w1(cz + loc_oz(a), loc_oz(A));
  return w;
}

// Output layout: entry-major, Ac[entry * mc + E]; thread t -> (entry = t / mc, E = t % mc), so
// the entry (and the constants it reads) is uniform within a warp.
template <int DIM, typename T>
__global__ void k_rap_from_fine(Dims df, const T* __restrict__ C, const T* __restrict__ x,
                                T* __restrict__ Ac, const double* __restrict__ g,
                                const double* __restrict__ Dinv) {
  pdl_prologue();
  constexpr int NN = DIM == 2 ? 4 : 8, NE = NN * DIM, NE2 = NE * NE;
  const int cnx = df.nx / 2, cny = df.ny / 2, cnz = DIM == 3 ? df.nz / 2 : 1;
  const long long mc = (long long)cnx * cny * cnz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= mc * NE2) return;
  const int entry = (int)(t / mc);
  const long long E = t % mc;
  const int EX = (int)(E % cnx), EY = (int)((E / cnx) % cny), EZ = (int)(E / ((long long)cnx * cny));
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < NN; ++c) {
    const int fx = 2 * EX + (c & 1), fy = 2 * EY + ((c >> 1) & 1), fz = 2 * EZ + (c >> 2);
    const long long fe = fx + (long long)df.nx * (fy + (long long)df.ny * (DIM == 3 ? fz : 0));
    acc = fma(x[fe], __ldg(C + c * NE2 + entry), acc);
    if (g) {  // FP64 solvers only (T = double)  // rank-one term (P_c^T g_c)_I (P_c^T g_c)_J / D_c
      const int I = entry / NE, J = entry % NE;
      const int A = I / DIM, al = I % DIM, B = J / DIM, be = J % DIM;
      double hI = 0.0, hJ = 0.0;
      for (int a = 0; a < NN; ++a) {
        hI = fma(wchild<DIM>(c, a, A), g[fe * NE + a * DIM + al], hI);
        hJ = fma(wchild<DIM>(c, a, B), g[fe * NE + a * DIM + be], hJ);
      }
      acc = (T)fma(hI * hJ, Dinv[fe], (double)acc);
    }
  }
  Ac[t] = acc;
}

// Second coarse level straight from the finest densities: A_E = sum_f x_f C2_f over the 4^dim fine
// elements f below E, with C2_f = W_f^T K0 W_f (W_f: composite interpolation from E's nodes to the
// nodes of f).  Entry-major output; thread t -> (entry = t / mc, E = t % mc).
template <int DIM, typename T>
__global__ void k_rap2_from_fine(Dims df, const T* __restrict__ C2, const T* __restrict__ x,
                                 T* __restrict__ Ac) {
  pdl_prologue();
  constexpr int NN = DIM == 2 ? 4 : 8, NE = NN * DIM, NE2 = NE * NE, NF = NN * NN;
  const int cnx = df.nx / 4, cny = df.ny / 4, cnz = DIM == 3 ? df.nz / 4 : 1;
  const long long mc = (long long)cnx * cny * cnz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= mc * NE2) return;
  const int entry = (int)(t / mc);
  const long long E = t % mc;
  const int EX = (int)(E % cnx), EY = (int)((E / cnx) % cny), EZ = (int)(E / ((long long)cnx * cny));
  T acc = T(0);
#pragma unroll 4
  for (int f = 0; f < NF; ++f) {
    const int c1 = f / NN, c2 = f % NN;
    const int fx = 4 * EX + 2 * (c1 & 1) + (c2 & 1);
    const int fy = 4 * EY + 2 * ((c1 >> 1) & 1) + ((c2 >> 1) & 1);
    const int fz = DIM == 3 ? 4 * EZ + 2 * (c1 >> 2) + (c2 >> 2) : 0;
    const long long fe = fx + (long long)df.nx * (fy + (long long)df.ny * fz);
    acc = fma(x[fe], __ldg(C2 + (long long)f * NE2 + entry), acc);
  }
  Ac[t] = acc;
}

// 1 / diag of the first coarse level straight from the finest densities:
// diag(A_1)_i = sum_{E at node} sum_c x_c (C_c)_{ii}.
template <int DIM, typename T>
__global__ void k_inv_diag_l1(Dims dc, const T* __restrict__ C, const T* __restrict__ xf,
                              const uint8_t* __restrict__ fixed, T* __restrict__ invd) {
  pdl_prologue();
  constexpr int NN = DIM == 2 ? 4 : 8, NE = NN * DIM, NE2 = NE * NE;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= dc.nodes()) return;
  const int nnx = dc.nx + 1, nny = dc.ny + 1;
  const int i = (int)(node % nnx), j = (int)((node / nnx) % nny);
  const int k = (DIM == 3) ? (int)(node / ((long long)nnx * nny)) : 0;
  const int fnx = 2 * dc.nx, fny = 2 * dc.ny;
  T acc[DIM] = {};
  for (int s = 0; s < NN; ++s) {
    const int dx = s & 1, dy = (s >> 1) & 1, dz = (DIM == 3) ? (s >> 2) : 0;
    const int ex = i - 1 + dx, ey = j - 1 + dy, ez = (DIM == 3) ? k - 1 + dz : 0;
    if (ex < 0 || ex >= dc.nx || ey < 0 || ey >= dc.ny) continue;
    if (DIM == 3 && (ez < 0 || ez >= dc.nz)) continue;
    const int loc = loc_of(1 - dx, 1 - dy, DIM == 3 ? 1 - dz : 0);
    for (int c = 0; c < NN; ++c) {
      const long long fe = (2 * ex + (c & 1)) +
                           (long long)fnx * ((2 * ey + ((c >> 1) & 1)) +
                                             (long long)fny * (DIM == 3 ? 2 * ez + (c >> 2) : 0));
      const T xc = xf[fe];
      for (int cc = 0; cc < DIM; ++cc) {
        const int r = loc * DIM + cc;
        acc[cc] = fma(xc, C[c * NE2 + r * NE + r], acc[cc]);
      }
    }
  }
  for (int cc = 0; cc < DIM; ++cc) {
    const long long id = DIM * node + cc;
    invd[id] = (fixed[id] || !(acc[cc] > T(0))) ? T(1) : T(1) / acc[cc];
  }
}

// General Galerkin step from level matrices Af (entry-major, mf elements) to Ac (entry-major):
// A_E = sum_c P_c^T A_c P_c with the interpolation weights W_c[a][A] tabulated in shared memory
// (exact binary fractions) and their zeros skipped.
template <int DIM, typename TI, typename TO>
__global__ void k_rap_coarse(Dims df, const TI* __restrict__ Af, TO* __restrict__ Ac) {
  pdl_prologue();
  constexpr int NN = DIM == 2 ? 4 : 8, NE = NN * DIM, NE2 = NE * NE;
  __shared__ float W[NN][NN][NN];  // [child][fine local node a][coarse local node A]
  for (int idx = threadIdx.x; idx < NN * NN * NN; idx += blockDim.x) {
    const int c = idx / (NN * NN), a = (idx / NN) % NN, A = idx % NN;
    W[c][a][A] = (float)wchild<DIM>(c, a, A);
  }
  __syncthreads();
  const int cnx = df.nx / 2, cny = df.ny / 2, cnz = DIM == 3 ? df.nz / 2 : 1;
  const long long mc = (long long)cnx * cny * cnz;
  const long long mf = df.elems();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= mc * NE2) return;
  const int entry = (int)(t / mc);
  const long long E = t % mc;
  const int I = entry / NE, J = entry % NE;
  const int A = I / DIM, al = I % DIM, B = J / DIM, be = J % DIM;
  const int EX = (int)(E % cnx), EY = (int)((E / cnx) % cny), EZ = (int)(E / ((long long)cnx * cny));
  TO acc = TO(0);
  for (int c = 0; c < NN; ++c) {
    const int fx = 2 * EX + (c & 1), fy = 2 * EY + ((c >> 1) & 1), fz = 2 * EZ + (c >> 2);
    const long long fe = fx + (long long)df.nx * (fy + (long long)df.ny * (DIM == 3 ? fz : 0));
    for (int a = 0; a < NN; ++a) {
      const float wa = W[c][a][A];
      if (wa == 0.0f) continue;
      TO s = TO(0);
      for (int b = 0; b < NN; ++b) {
        const float wb = W[c][b][B];
        if (wb == 0.0f) continue;
        s = fma((TO)__ldg(Af + (long long)((a * DIM + al) * NE + b * DIM + be) * mf + fe), (TO)wb, s);
      }
      acc = fma((TO)wa, s, acc);
    }
  }
  Ac[t] = acc;
}

// ---- 2D Galerkin products, one thread per coarse element ----------------------------------
// The entry-parallel kernels above re-read each fine value once per output entry that uses it
// (16 to 64 times) and spend most of their instructions on index arithmetic and zero-weight
// tests.  In 2D one thread can hold all 64 outputs of its coarse element; the weights are then
// compile-time constants (the zero ones vanish from the code), every fine value is read once,
// and the constant tables travel in the kernel's parameter space, so each multiply-add reads its
// table operand from the constant bank.  Every output is accumulated in the same order as in the
// entry-parallel kernels (the same bits).

template <typename T, int N>
struct ConstTable {
  T v[N];
};

__host__ __device__ constexpr float w1c(int p, int q) {
  return (p - 2 * q == 0) ? 1.0f : ((p - 2 * q == 1 || p - 2 * q == -1) ? 0.5f : 0.0f);
}
__host__ __device__ constexpr int lox(int a) { return ((a & 3) == 1 || (a & 3) == 2) ? 1 : 0; }
__host__ __device__ constexpr int loy(int a) { return ((a & 3) >= 2) ? 1 : 0; }
// wchild<2>(c, a, A) as a constant expression
__host__ __device__ constexpr float w2c(int c, int a, int A) {
  return w1c((c & 1) + lox(a), lox(A)) * w1c(((c >> 1) & 1) + loy(a), loy(A));
}

constexpr int kRapElemThreads = 128;

// One thread per coarse element pays where its outputs are FP32, or where the coarse level has
// enough elements to fill the GPU; FP64 outputs of a small level (a few thousand elements or
// fewer: the coarsest levels, the small IP hierarchies) are FP64-bound and want one thread per
// output entry.
template <typename TO>
bool rap_elem_parallel(long long mc) {
  return std::is_same<TO, float>::value || mc >= 152LL * kRapElemThreads;
}

// First coarse level (k_rap_from_fine, 2D): A_E = sum_c x_c C_c (+ rank-one terms of Z).
template <typename T>
__global__ void __launch_bounds__(kRapElemThreads)
    k_rap1_elem2d(Dims df, const __grid_constant__ ConstTable<T, 256> C, const T* __restrict__ x,
                  T* __restrict__ Ac, const double* __restrict__ g,
                  const double* __restrict__ Dinv) {
  pdl_prologue();
  const int cnx = df.nx / 2, cny = df.ny / 2;
  const long long mc = (long long)cnx * cny;
  const long long E = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (E >= mc) return;
  const int EX = (int)(E % cnx), EY = (int)(E / cnx);
  T acc[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) acc[q] = T(0);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const long long fe = (2 * EX + (c & 1)) + (long long)df.nx * (2 * EY + ((c >> 1) & 1));
    const T xc = x[fe];
#pragma unroll
    for (int q = 0; q < 64; ++q) acc[q] = fma(xc, C.v[c * 64 + q], acc[q]);
    if (g) {
      double gc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) gc[q] = g[fe * 8 + q];
      const double dc = Dinv[fe];
      double h[8];
#pragma unroll
      for (int I = 0; I < 8; ++I) {
        double hv = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a) hv = fma((double)w2c(c, a, I / 2), gc[a * 2 + I % 2], hv);
        h[I] = hv;
      }
#pragma unroll
      for (int q = 0; q < 64; ++q) acc[q] = (T)fma(h[q / 8] * h[q % 8], dc, (double)acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 64; ++q) Ac[q * mc + E] = acc[q];
}

// Second coarse level from the finest densities (k_rap2_from_fine, 2D): A_E = sum_f x_f C2_f.
template <typename T>
__global__ void __launch_bounds__(kRapElemThreads)
    k_rap2_elem2d(Dims df, const __grid_constant__ ConstTable<T, 1024> C2,
                  const T* __restrict__ x, T* __restrict__ Ac) {
  pdl_prologue();
  const int cnx = df.nx / 4, cny = df.ny / 4;
  const long long mc = (long long)cnx * cny;
  const long long E = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (E >= mc) return;
  const int EX = (int)(E % cnx), EY = (int)(E / cnx);
  T xf[16];
#pragma unroll
  for (int f = 0; f < 16; ++f) {
    const int c1 = f / 4, c2 = f % 4;
    const int fx = 4 * EX + 2 * (c1 & 1) + (c2 & 1);
    const int fy = 4 * EY + 2 * ((c1 >> 1) & 1) + ((c2 >> 1) & 1);
    xf[f] = x[fx + (long long)df.nx * fy];
  }
#pragma unroll
  for (int q = 0; q < 64; ++q) {
    T acc = T(0);
#pragma unroll
    for (int f = 0; f < 16; ++f) acc = fma(xf[f], C2.v[f * 64 + q], acc);
    Ac[q * mc + E] = acc;
  }
}

// Deeper levels (k_rap_coarse, 2D): A_E = sum_c P_c^T A_c P_c, row pair (a, 0..1) of each child
// read once and applied to every output it feeds.
template <typename TI, typename TO>
__global__ void __launch_bounds__(kRapElemThreads)
    k_rap_coarse_elem2d(Dims df, const TI* __restrict__ Af, TO* __restrict__ Ac) {
  pdl_prologue();
  const int cnx = df.nx / 2, cny = df.ny / 2;
  const long long mc = (long long)cnx * cny;
  const long long mf = df.elems();
  const long long E = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (E >= mc) return;
  const int EX = (int)(E % cnx), EY = (int)(E / cnx);
  TO acc[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) acc[q] = TO(0);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const long long fe = (2 * EX + (c & 1)) + (long long)df.nx * (2 * EY + ((c >> 1) & 1));
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      TO row[2][8];
#pragma unroll
      for (int al = 0; al < 2; ++al)
#pragma unroll
        for (int q = 0; q < 8; ++q)
          row[al][q] = (TO)__ldg(Af + (long long)((a * 2 + al) * 8 + q) * mf + fe);
#pragma unroll
      for (int A = 0; A < 4; ++A) {
        constexpr float kZero = 0.0f;
        const float wa = w2c(c, a, A);
        if (wa == kZero) continue;
#pragma unroll
        for (int al = 0; al < 2; ++al)
#pragma unroll
          for (int J = 0; J < 8; ++J) {
            const int B = J / 2, be = J % 2;
            TO sv = TO(0);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const float wb = w2c(c, b, B);
              if (wb == kZero) continue;
              sv = fma(row[al][b * 2 + be], (TO)wb, sv);
            }
            acc[(A * 2 + al) * 8 + J] = fma((TO)wa, sv, acc[(A * 2 + al) * 8 + J]);
          }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 64; ++q) Ac[q * mc + E] = acc[q];
}

// Dense operator of a level (used for the coarsest level): entry (i, j) gathers the elements that
// hold both DOFs' nodes.  Fixed DOFs get identity rows and columns.
template <int DIM>
__global__ void k_assemble_dense(Dims d, const double* __restrict__ K0,
                                 const double* __restrict__ x, const double* __restrict__ Ae,
                                 const uint8_t* __restrict__ fixed, double* __restrict__ A,
                                 long long ld, const double* __restrict__ w,
                                 const double* __restrict__ zll, const double* __restrict__ g,
                                 const double* __restrict__ Dinv) {
  pdl_prologue();
  constexpr int NE = (DIM == 2 ? 4 : 8) * DIM;
  const long long n = d.dofs();
  const long long na = w ? n + 1 : n;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= na * na) return;
  const long long i = t / na, j = t % na;
  double* out = A + i * ld + j;
  if (i == n || j == n) {  // arrow row / column
    if (i == n && j == n) *out = *zll;
    else {
      const long long k = (i == n) ? j : i;
      *out = fixed[k] ? 0.0 : w[k];
    }
    return;
  }
  if (fixed[i] || fixed[j]) {
    *out = (i == j) ? 1.0 : 0.0;
    return;
  }
  const int nnx = d.nx + 1, nny = d.ny + 1;
  const long long ni = i / DIM, nj = j / DIM;
  const int al = (int)(i % DIM), be = (int)(j % DIM);
  const int xi = (int)(ni % nnx), yi = (int)((ni / nnx) % nny), zi = (int)(ni / ((long long)nnx * nny));
  const int xj = (int)(nj % nnx), yj = (int)((nj / nnx) % nny), zj = (int)(nj / ((long long)nnx * nny));
  double acc = 0.0;
  for (int s = 0; s < (DIM == 2 ? 4 : 8); ++s) {
    const int ex = xi - 1 + (s & 1), ey = yi - 1 + ((s >> 1) & 1), ez = DIM == 3 ? zi - 1 + (s >> 2) : 0;
    if (ex < 0 || ex >= d.nx || ey < 0 || ey >= d.ny) continue;
    if (DIM == 3 && (ez < 0 || ez >= d.nz)) continue;
    const int lxj = xj - ex, lyj = yj - ey, lzj = DIM == 3 ? zj - ez : 0;
    if (lxj < 0 || lxj > 1 || lyj < 0 || lyj > 1 || lzj < 0 || lzj > 1) continue;
    const int li = loc_of(xi - ex, yi - ey, DIM == 3 ? zi - ez : 0);
    const int lj = loc_of(lxj, lyj, lzj);
    const long long e = ex + (long long)d.nx * (ey + (long long)d.ny * ez);
    const int r = li * DIM + al, q = lj * DIM + be;
    acc += x ? x[e] * K0[r * NE + q] : Ae[(long long)(r * NE + q) * d.elems() + e];
    if (x && g) acc += g[e * NE + r] * g[e * NE + q] * Dinv[e];
  }
  *out = acc;
}

// Pivots that rounding has pushed to or below kPivotFloor times the original diagonal entry are
// raised to that floor (a modified Cholesky): the coarsest solve stays an SPD preconditioner when
// the Schur complement of the IP multiplier cancels to rounding level in late interior-point steps.
constexpr double kPivotFloor = 1e-13;

// In-place Cholesky A = L L^T of a dense SPD matrix in one block (right-looking), then L^T is
// mirrored into the strict upper triangle.  info = 0, or k+1 if the k-th diagonal entry is not
// positive or a pivot is not finite.
__global__ void __launch_bounds__(1024) k_cholesky(int n, double* A, double* diag0, int* info,
                                                  const int* only_if) {
  pdl_prologue();
  if (only_if && !*only_if) return;  // Newton-Schulz inverse already accepted
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) diag0[k] = A[(long long)k * n + k];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      double akk = A[(long long)k * n + k];
      const double a0 = diag0[k];
      if (!(a0 > 0.0) || !isfinite(akk)) bad = k + 1;
      else A[(long long)k * n + k] = sqrt(fmax(akk, kPivotFloor * a0));
    }
    __syncthreads();
    if (bad) break;
    const double lkk = A[(long long)k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(long long)i * n + k] /= lkk;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = k + 1 + warp; i < n; i += nw) {
      const double lik = A[(long long)i * n + k];
      for (int j = k + 1 + lane; j <= i; j += 32)
        A[(long long)i * n + j] -= lik * A[(long long)j * n + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *info = bad;
  if (bad) return;
  for (long long idx = threadIdx.x; idx < (long long)n * n; idx += blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    if (j > i) A[idx] = A[(long long)j * n + i];
  }
}

// Row j of A^{-1} = solution of A w = e_j with the factor (L lower, L^T upper): one warp per row,
// the row being built kept in shared memory (kInvWarps warps per block, n <= kMaxCoarse).
constexpr int kInvWarps = 8;

inline int inv_warps(int n) {
  const int w = (int)((200 * 1024) / ((size_t)n * sizeof(double)));
  return w < 1 ? 1 : (w > kInvWarps ? kInvWarps : w);
}

__global__ void __launch_bounds__(kInvWarps * 32) k_chol_inverse(int n, const double* __restrict__ LU,
                                                                 double* Ainv, const int* info,
                                                                 const int* only_if) {
  pdl_prologue();
  extern __shared__ double wsh[];  // [warps per block][n]
  if (*info || (only_if && !*only_if)) return;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + wib;
  if (j >= n) return;
  double* w = wsh + (long long)wib * n;
  for (int k = lane; k < n; k += 32) w[k] = 0.0;
  __syncwarp();
  for (int i = j; i < n; ++i) {  // forward: L w = e_j
    const double* Li = LU + (long long)i * n;
    double s = 0.0;
    for (int k = j + lane; k < i; k += 32) s = fma(__ldg(Li + k), w[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[i] = ((i == j ? 1.0 : 0.0) - s) / __ldg(Li + i);
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {  // backward: L^T w = y
    const double* Ui = LU + (long long)i * n;
    double s = 0.0;
    for (int k = i + 1 + lane; k < n; k += 32) s = fma(__ldg(Ui + k), w[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[i] = (w[i] - s) / __ldg(Ui + i);
    __syncwarp();
  }
  double* out = Ainv + (long long)j * n;
  for (int k = lane; k < n; k += 32) out[k] = w[k];
}

// Cholesky in shared memory for small n (n * n doubles fit in one block's shared memory).
__global__ void __launch_bounds__(1024) k_cholesky_smem(int n, double* A, double* diag0, int* info,
                                                       const int* only_if) {
  pdl_prologue();
  if (only_if && !*only_if) return;  // Newton-Schulz inverse already accepted
  extern __shared__ double S[];
  __shared__ int bad;
  const long long nn = (long long)n * n;
  for (long long t = threadIdx.x; t < nn; t += blockDim.x) S[t] = A[t];
  for (int k = threadIdx.x; k < n; k += blockDim.x) diag0[k] = A[(long long)k * n + k];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double akk = S[k * n + k];
      const double a0 = diag0[k];
      if (!(a0 > 0.0) || !isfinite(akk)) bad = k + 1;
      else S[k * n + k] = sqrt(fmax(akk, kPivotFloor * a0));
    }
    __syncthreads();
    if (bad) break;
    const double lkk = S[k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) S[i * n + k] /= lkk;
    __syncthreads();
    for (int i = k + 1 + warp; i < n; i += nw) {
      const double lik = S[i * n + k];
      for (int jj = k + 1 + lane; jj <= i; jj += 32) S[i * n + jj] -= lik * S[jj * n + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *info = bad;
  if (bad) return;
  for (long long t = threadIdx.x; t < nn; t += blockDim.x) {
    const int i = (int)(t / n), jj = (int)(t % n);
    A[t] = (jj > i) ? S[(long long)jj * n + i] : S[t];
  }
}

// Small coarsest matrices (n <= kGjMaxN) are inverted without an FP64 factorisation, whose n
// dependent steps run at the FP64 rate of a single SM: a Gauss-Jordan inverse in FP32 in one
// block gives X0, and Newton-Schulz steps X <- X (2I - A X) in FP64, each two n x n products
// spread over n blocks, square the error ||I - A X|| until it is at FP64 rounding.  The last
// step checks ||I - A X||_max <= kNsTol before its product; above it (or not finite) the flag
// is set and the Cholesky path below recomputes the inverse from A.
constexpr int kGjMaxN = 128;
constexpr int kNsSteps = 4;
constexpr double kNsTol = 1e-7;

// Gauss-Jordan step k with pivot p maps a_kk -> 1/p, a_kj -> a_kj/p, a_ik -> -a_ik/p and
// a_ij -> a_ij - a_ik a_kj / p (old values on the right); after n steps the array holds A^{-1}.
// No pivoting: the pivots of an SPD matrix are its Schur-complement diagonals.  512 threads: lane
// tx and warp ty keep the EA x EB entries (ty + 16a, tx + 32b), EA = ceil(n / 16), EB = ceil(n / 32),
// in registers.  A step is one multiply-add per entry (the general update), then the threads that
// hold row k (one warp row) and column k (one lane) overwrite them with the old row times 1/p (the
// old row is the staged pivot row) and -a_ik/p, and the holders of row and column k + 1 stage them
// for the next step in double-buffered shared arrays: one barrier per step, registers indexed by
// constants only.  (The per-entry branches or selects of the special cases, with 1024 or 256
// threads, took 108-119 us for n = 90: about 415 dependent instructions per warp and step.)  Also
// clears info[0] and the Newton-Schulz flag.
constexpr int kGjLanes = 32, kGjRows = 16;

template <int EA>
__global__ void __launch_bounds__(kGjLanes * kGjRows) k_gj32_start(int n,
                                                                   const double* __restrict__ A,
                                                                   double* __restrict__ X,
                                                                   int* info, int* ns_bad) {
  constexpr int EB = (EA + 1) / 2;  // (n <= 16 EA gives ceil(n / 32) <= EB)
  pdl_prologue();
  __shared__ float Pb[2][kGjMaxN];  // pivot row (values before the step), by step parity
  __shared__ float Cb[2][kGjMaxN];  // pivot column (values before the step), by step parity
  const int tx = threadIdx.x % kGjLanes, ty = threadIdx.x / kGjLanes;
  if (threadIdx.x == 0) {
    *info = 0;
    *ns_bad = 0;
  }
  float r[EA][EB];
#pragma unroll
  for (int a = 0; a < EA; ++a)
#pragma unroll
    for (int b = 0; b < EB; ++b) {
      const int i = ty + kGjRows * a, j = tx + kGjLanes * b;
      const bool in = i < n && j < n;
      r[a][b] = in ? (float)A[(long long)i * n + j] : 0.0f;
      if (in && j == 0) Cb[0][i] = r[a][b];
      if (in && i == 0) Pb[0][j] = r[a][b];
    }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const int cur = k & 1;
    const float rp = 1.0f / Pb[cur][k];
    float pj[EB], fi[EA];
#pragma unroll
    for (int b = 0; b < EB; ++b)
      pj[b] = (tx + kGjLanes * b < n) ? Pb[cur][tx + kGjLanes * b] : 0.0f;
#pragma unroll
    for (int a = 0; a < EA; ++a)
      fi[a] = (ty + kGjRows * a < n) ? Cb[cur][ty + kGjRows * a] * rp : 0.0f;
#pragma unroll
    for (int a = 0; a < EA; ++a)
#pragma unroll
      for (int b = 0; b < EB; ++b) r[a][b] = fmaf(-fi[a], pj[b], r[a][b]);
    // (selects over every entry held, inside branches taken only by the holders: an indexed
    // store of the same update would move the register array to local memory)
    const int kb = k / kGjLanes, ka = k / kGjRows;
    if (tx == k % kGjLanes) {  // column k: -a_ik / p
#pragma unroll
      for (int a = 0; a < EA; ++a)
#pragma unroll
        for (int b = 0; b < EB; ++b) r[a][b] = (b == kb) ? -fi[a] : r[a][b];
    }
    if (ty == k % kGjRows) {  // row k: a_kj / p, and 1 / p on the diagonal
#pragma unroll
      for (int a = 0; a < EA; ++a)
#pragma unroll
        for (int b = 0; b < EB; ++b) {
          const float rowv = (tx + kGjLanes * b == k) ? rp : pj[b] * rp;
          r[a][b] = (a == ka) ? rowv : r[a][b];
        }
    }
    const int k1 = k + 1;  // stage row and column k + 1 for the next step
    if (k1 < n) {
      float* Pn = Pb[cur ^ 1];
      float* Cn = Cb[cur ^ 1];
      const int kb1 = k1 / kGjLanes, ka1 = k1 / kGjRows;
      if (ty == k1 % kGjRows) {
#pragma unroll
        for (int b = 0; b < EB; ++b) {
          float v = 0.0f;
#pragma unroll
          for (int a = 0; a < EA; ++a) v = (a == ka1) ? r[a][b] : v;
          if (tx + kGjLanes * b < n) Pn[tx + kGjLanes * b] = v;
        }
      }
      if (tx == k1 % kGjLanes) {
#pragma unroll
        for (int a = 0; a < EA; ++a) {
          float v = 0.0f;
#pragma unroll
          for (int b = 0; b < EB; ++b) v = (b == kb1) ? r[a][b] : v;
          if (ty + kGjRows * a < n) Cn[ty + kGjRows * a] = v;
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < EA; ++a)
#pragma unroll
    for (int b = 0; b < EB; ++b) {
      const int i = ty + kGjRows * a, j = tx + kGjLanes * b;
      if (i < n && j < n) X[(long long)i * n + j] = (double)r[a][b];
    }
}

// C = alpha I + beta L R for n x n matrices: an 8 x 8 tile of C per block of 64 threads (about
// 150 blocks for n = 90, so that the FP64 multiply-adds, 2 per clock on an SM, spread over the
// GPU); the tile's rows of L and columns of R are staged in shared memory, and each entry sums
// over k in increasing order from zero (the arithmetic of one dot product per entry; a form with
// one block per row of C took 8.9 us per product for n = 90).  check: set *bad if some
// |C_ij - delta_ij| > kNsTol or is not finite (C = 2I - A X gives I - A X).
constexpr int kNsTile = 8;

__global__ void __launch_bounds__(kNsTile * kNsTile) k_ns_gemm(int n, const double* __restrict__ L,
                                                               const double* __restrict__ R,
                                                               double* __restrict__ C,
                                                               double alpha, double beta, int check,
                                                               int* bad) {
  pdl_prologue();
  __shared__ double Ls[kNsTile][kGjMaxN];  // rows i0 .. i0 + 7 of L
  __shared__ double Rs[kGjMaxN][kNsTile];  // columns j0 .. j0 + 7 of R
  const int i0 = blockIdx.y * kNsTile, j0 = blockIdx.x * kNsTile;
  // every load of the tile in flight at once, then the stores (one L2 round trip)
  constexpr int kPer = kNsTile * kGjMaxN / (kNsTile * kNsTile);
  double lv[kPer], rv[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int q = threadIdx.x + u * kNsTile * kNsTile;
    lv[u] = rv[u] = 0.0;
    if (q < kNsTile * n) {
      const int a = q / n, k = q - a * n;  // (row-major reads of L's rows)
      if (i0 + a < n) lv[u] = L[(long long)(i0 + a) * n + k];
      const int kk = q / kNsTile, b = q - kk * kNsTile;  // (R's rows, 8 columns each)
      if (j0 + b < n) rv[u] = R[(long long)kk * n + j0 + b];
    }
  }
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int q = threadIdx.x + u * kNsTile * kNsTile;
    if (q < kNsTile * n) {
      const int a = q / n, k = q - a * n;
      Ls[a][k] = lv[u];
      const int kk = q / kNsTile, b = q - kk * kNsTile;
      Rs[kk][b] = rv[u];
    }
  }
  __syncthreads();
  const int ti = threadIdx.x / kNsTile, tj = threadIdx.x % kNsTile;
  const int i = i0 + ti, j = j0 + tj;
  if (i >= n || j >= n) return;
  double acc = 0.0;
#pragma unroll 8
  for (int k = 0; k < n; ++k) acc = fma(Ls[ti][k], Rs[k][tj], acc);
  const double c = fma(beta, acc, i == j ? alpha : 0.0);
  C[(long long)i * n + j] = c;
  if (check && !(fabs(c - (i == j ? 1.0 : 0.0)) <= kNsTol)) atomicOr(bad, 1);
}

// Larger coarsest matrices (n > kGjMaxN: 3D grids, the IP systems' 2D coarsest levels) are
// inverted by block Gauss-Jordan in FP64 on tiles of kBg x kBg over many blocks: an n-step
// factorisation on one SM runs at the FP64 rate of that SM alone (21 ms for n = 675).  The matrix
// is padded with the identity to a multiple of kBg.  Block step K, with P = W_KK^{-1} formed by
// scalar Gauss-Jordan (the pivots are the same Schur-complement diagonals as in the scalar
// elimination, so the same floor and failure test apply):
//   Z_J = P W_KJ (J != K);  W_IJ -= W_IK Z_J (I, J != K);  W_IK <- -W_IK P, W_KJ <- Z_J, W_KK <- P.
// After the last step W holds the inverse.
constexpr int kBg = 32;

// W (npad x npad) = [A 0; 0 I], a0 = diagonal of A (1 on the padding).
__global__ void k_bgj_setup(int n, int npad, const double* __restrict__ A, double* __restrict__ W,
                            double* __restrict__ a0, int* info) {
  pdl_prologue();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) *info = 0;
  if (t >= (long long)npad * npad) return;
  const int i = (int)(t / npad), j = (int)(t % npad);
  const double v = (i < n && j < n) ? A[(long long)i * n + j] : (i == j ? 1.0 : 0.0);
  W[t] = v;
  if (i == j) a0[i] = v;
}

// P = W_KK^{-1} by scalar Gauss-Jordan in shared memory (one block of kBg * 8 threads, each
// thread 4 entries of the tile); pivot floor and failure test as in the Cholesky kernels.
__global__ void __launch_bounds__(kBg * 8) k_bgj_pivot(int npad, int K, const double* __restrict__ W,
                                                       const double* __restrict__ a0,
                                                       double* __restrict__ P, int* info) {
  pdl_prologue();
  // Two copies of the tile (step k reads one and writes the other) and the pivot reciprocal of
  // each step, formed by the thread that writes the next pivot entry: one barrier per step.
  __shared__ double S[2][kBg][kBg + 1];
  __shared__ double D0[kBg];
  __shared__ double rp_s[2];
  __shared__ int bad_s[2];
  const int tid = threadIdx.x;
  const long long base = (long long)K * kBg;
  for (int t = tid; t < kBg * kBg; t += blockDim.x)
    S[0][t / kBg][t % kBg] = W[(base + t / kBg) * npad + base + t % kBg];
  if (tid < kBg) D0[tid] = a0[base + tid];
  __syncthreads();
  // pivot k: floored at kPivotFloor times the original diagonal (a non-positive original
  // diagonal or a non-finite entry marks the matrix as not positive definite).  Slot k & 1 is
  // written during step k - 1 and read after its barrier; step k - 1 read the other slot.
  auto pivot = [&](int k, double akk) {
    const double d0 = D0[k];
    bad_s[k & 1] = (!(d0 > 0.0) || !isfinite(akk)) ? 1 : 0;
    rp_s[k & 1] = 1.0 / fmax(akk, kPivotFloor * d0);
  };
  if (tid == 0) pivot(0, S[0][0][0]);
  __syncthreads();
  int cur = 0;
  bool bad = false;
  for (int k = 0; k < kBg; ++k) {
    if (bad_s[k & 1]) {  // the same value in every thread
      bad = true;
      break;
    }
    const double rp = rp_s[k & 1];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int t = tid + r * blockDim.x;
      const int i = t / kBg, j = t % kBg;
      const double aij = S[cur][i][j];
      double nv;
      if (i == k) nv = (j == k) ? rp : aij * rp;
      else if (j == k) nv = -aij * rp;
      else nv = fma(-S[cur][i][k] * rp, S[cur][k][j], aij);
      S[cur ^ 1][i][j] = nv;
      if (k + 1 < kBg && i == k + 1 && j == k + 1) pivot(k + 1, nv);
    }
    cur ^= 1;
    __syncthreads();
  }
  if (bad) {
    if (tid == 0 && *info == 0) {
      int k = 0;  // first failing pivot of this block, for the report
      while (k < kBg && a0[base + k] > 0.0) ++k;
      *info = (int)(base + (k < kBg ? k : 0)) + 1;
    }
    return;
  }
  for (int t = tid; t < kBg * kBg; t += blockDim.x) P[t] = S[cur][t / kBg][t % kBg];
}

// C = X Y for kBg x kBg tiles in shared memory; each of the kBg * 8 threads forms 4 outputs.
__device__ __forceinline__ void tile_mm(const double (*X)[kBg + 1], const double (*Y)[kBg + 1],
                                        double out[4]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int t = tid + r * blockDim.x;
    const int i = t / kBg, j = t % kBg;
    double acc = 0.0;
#pragma unroll 8
    for (int l = 0; l < kBg; ++l) acc = fma(X[i][l], Y[l][j], acc);
    out[r] = acc;
  }
}

// Z_J = P W_KJ for every tile column J != K (block J).
__global__ void __launch_bounds__(kBg * 8) k_bgj_zrow(int npad, int K, const double* __restrict__ W,
                                                      const double* __restrict__ P,
                                                      double* __restrict__ Z, const int* info) {
  pdl_prologue();
  if (*info) return;
  const int J = blockIdx.x;
  if (J == K) return;
  __shared__ double Ps[kBg][kBg + 1], Bs[kBg][kBg + 1];
  const long long rb = (long long)K * kBg, cb = (long long)J * kBg;
  for (int t = threadIdx.x; t < kBg * kBg; t += blockDim.x) {
    Ps[t / kBg][t % kBg] = P[t];
    Bs[t / kBg][t % kBg] = W[(rb + t / kBg) * npad + cb + t % kBg];
  }
  __syncthreads();
  double out[4];
  tile_mm(Ps, Bs, out);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int t = threadIdx.x + r * blockDim.x;
    Z[(long long)(t / kBg) * npad + cb + t % kBg] = out[r];
  }
}

// W_IJ -= W_IK Z_J for I, J != K (block (J, I)).
__global__ void __launch_bounds__(kBg * 8) k_bgj_update(int npad, int K, double* __restrict__ W,
                                                        const double* __restrict__ Z,
                                                        const int* info) {
  pdl_prologue();
  if (*info) return;
  const int J = blockIdx.x, I = blockIdx.y;
  if (I == K || J == K) return;
  __shared__ double As[kBg][kBg + 1], Zs[kBg][kBg + 1];
  const long long ib = (long long)I * kBg, jb = (long long)J * kBg, kb = (long long)K * kBg;
  for (int t = threadIdx.x; t < kBg * kBg; t += blockDim.x) {
    As[t / kBg][t % kBg] = W[(ib + t / kBg) * npad + kb + t % kBg];
    Zs[t / kBg][t % kBg] = Z[(long long)(t / kBg) * npad + jb + t % kBg];
  }
  __syncthreads();
  double out[4];
  tile_mm(As, Zs, out);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int t = threadIdx.x + r * blockDim.x;
    double* w = W + (ib + t / kBg) * npad + jb + t % kBg;
    *w = *w - out[r];
  }
}

// W_IK <- -W_IK P, W_KI <- Z_I (block I != K); W_KK <- P (block K).
__global__ void __launch_bounds__(kBg * 8) k_bgj_final(int npad, int K, double* __restrict__ W,
                                                       const double* __restrict__ P,
                                                       const double* __restrict__ Z,
                                                       const int* info) {
  pdl_prologue();
  if (*info) return;
  const int I = blockIdx.x;
  const long long ib = (long long)I * kBg, kb = (long long)K * kBg;
  if (I == K) {
    for (int t = threadIdx.x; t < kBg * kBg; t += blockDim.x)
      W[(kb + t / kBg) * npad + kb + t % kBg] = P[t];
    return;
  }
  __shared__ double As[kBg][kBg + 1], Ps[kBg][kBg + 1];
  for (int t = threadIdx.x; t < kBg * kBg; t += blockDim.x) {
    As[t / kBg][t % kBg] = W[(ib + t / kBg) * npad + kb + t % kBg];
    Ps[t / kBg][t % kBg] = P[t];
  }
  __syncthreads();
  double out[4];
  tile_mm(As, Ps, out);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int t = threadIdx.x + r * blockDim.x;
    W[(ib + t / kBg) * npad + kb + t % kBg] = -out[r];
    W[(kb + t / kBg) * npad + ib + t % kBg] = Z[(long long)(t / kBg) * npad + ib + t % kBg];
  }
}

// Ainv (n x n) = the leading block of W.
__global__ void k_bgj_copy(int n, int npad, const double* __restrict__ W, double* __restrict__ Ainv,
                           const int* info) {
  pdl_prologue();
  if (*info) return;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  Ainv[t] = W[(t / n) * npad + t % n];
}

// z = A^{-1} b: one warp per row; FP64 accumulation for FP64 vectors, float-pair accumulation with
// Ainv as pairs for FP32 vectors (AinvDF).
template <typename T>
__global__ void k_dense_solve(int n, const double* __restrict__ Ainv,
                              const float2* __restrict__ AinvDF, const T* __restrict__ b,
                              T* __restrict__ z, const CgScalars* __restrict__ sc) {
  pdl_prologue();
  const int rhs = blockIdx.y;
  if (sc && sc[rhs].done) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  b += (long long)rhs * n;
  z += (long long)rhs * n;
  if constexpr (sizeof(T) == 4) {
    const f2 s = dense_row_dot_df<false>(n, AinvDF + (long long)warp * n, b, lane);
    if (lane == 0) z[warp] = __fadd_rn(s.h, s.l);
  } else {
    const double s = dense_row_dot<false>(n, Ainv + (long long)warp * n, b, lane);
    if (lane == 0) z[warp] = (T)s;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_rap_from_fine(const Dims& fine, const T* C, const T* x, T* Ac, cudaStream_t st,
                                 const double* g, const double* Dinv, const double* Ch) {
  const int ne = fine.dim == 2 ? 8 : 24;
  const long long mc = fine.elems() / (fine.dim == 2 ? 4 : 8);
  const long long total = mc * ne * ne;
  if (fine.dim == 2 && Ch && rap_elem_parallel<T>(mc)) {
    ConstTable<T, 256> tab;
    for (int i = 0; i < 256; ++i) tab.v[i] = (T)Ch[i];
    topo::launch(k_rap1_elem2d<T>, (unsigned)((mc + kRapElemThreads - 1) / kRapElemThreads),
                 kRapElemThreads, 0, st, fine, tab, x, Ac, g, Dinv);
  } else if (fine.dim == 2)
    topo::launch(k_rap_from_fine<2, T>, blocks_for(total), kThreads, 0, st, fine, C, x, Ac, g, Dinv);
  else
    topo::launch(k_rap_from_fine<3, T>, blocks_for(total), kThreads, 0, st, fine, C, x, Ac, g, Dinv);
  return cudaGetLastError();
}
template cudaError_t launch_rap_from_fine<double>(const Dims&, const double*, const double*,
                                                  double*, cudaStream_t, const double*,
                                                  const double*, const double*);
template cudaError_t launch_rap_from_fine<float>(const Dims&, const float*, const float*, float*,
                                                 cudaStream_t, const double*, const double*,
                                                 const double*);

template <typename T>
cudaError_t launch_rap2_from_fine(const Dims& fine, const T* C2, const T* x, T* Ac,
                                  cudaStream_t st, const double* C2h) {
  const int ne = fine.dim == 2 ? 8 : 24;
  const long long mc = fine.elems() / (fine.dim == 2 ? 16 : 64);
  const long long total = mc * ne * ne;
  if (fine.dim == 2 && C2h && rap_elem_parallel<T>(mc)) {
    ConstTable<T, 1024> tab;
    for (int i = 0; i < 1024; ++i) tab.v[i] = (T)C2h[i];
    topo::launch(k_rap2_elem2d<T>, (unsigned)((mc + kRapElemThreads - 1) / kRapElemThreads),
                 kRapElemThreads, 0, st, fine, tab, x, Ac);
  } else if (fine.dim == 2)
    topo::launch(k_rap2_from_fine<2, T>, blocks_for(total), kThreads, 0, st, fine, C2, x, Ac);
  else
    topo::launch(k_rap2_from_fine<3, T>, blocks_for(total), kThreads, 0, st, fine, C2, x, Ac);
  return cudaGetLastError();
}
template cudaError_t launch_rap2_from_fine<double>(const Dims&, const double*, const double*,
                                                   double*, cudaStream_t, const double*);
template cudaError_t launch_rap2_from_fine<float>(const Dims&, const float*, const float*, float*,
                                                  cudaStream_t, const double*);

template <typename T>
cudaError_t launch_inv_diag_l1(const Dims& coarse1, const T* C, const T* xf,
                               const uint8_t* fixed, T* invd, cudaStream_t st) {
  if (coarse1.dim == 2)
    topo::launch(k_inv_diag_l1<2, T>, blocks_for(coarse1.nodes()), kThreads, 0, st, coarse1, C, xf,
                 fixed, invd);
  else
    topo::launch(k_inv_diag_l1<3, T>, blocks_for(coarse1.nodes()), kThreads, 0, st, coarse1, C, xf,
                 fixed, invd);
  return cudaGetLastError();
}
template cudaError_t launch_inv_diag_l1<double>(const Dims&, const double*, const double*,
                                                const uint8_t*, double*, cudaStream_t);
template cudaError_t launch_inv_diag_l1<float>(const Dims&, const float*, const float*,
                                               const uint8_t*, float*, cudaStream_t);

template <typename TI, typename TO>
cudaError_t launch_rap_coarse(const Dims& fine, const TI* Af, TO* Ac, cudaStream_t st) {
  const int ne = fine.dim == 2 ? 8 : 24;
  const long long mc = fine.elems() / (fine.dim == 2 ? 4 : 8);
  const long long total = mc * ne * ne;
  if (fine.dim == 2 && rap_elem_parallel<TO>(mc))
    topo::launch(k_rap_coarse_elem2d<TI, TO>,
                 (unsigned)((mc + kRapElemThreads - 1) / kRapElemThreads), kRapElemThreads, 0, st,
                 fine, Af, Ac);
  else if (fine.dim == 2)
    topo::launch(k_rap_coarse<2, TI, TO>, blocks_for(total), kThreads, 0, st, fine, Af, Ac);
  else
    topo::launch(k_rap_coarse<3, TI, TO>, blocks_for(total), kThreads, 0, st, fine, Af, Ac);
  return cudaGetLastError();
}
template cudaError_t launch_rap_coarse<double, double>(const Dims&, const double*, double*,
                                                       cudaStream_t);
template cudaError_t launch_rap_coarse<float, float>(const Dims&, const float*, float*,
                                                     cudaStream_t);
template cudaError_t launch_rap_coarse<float, double>(const Dims&, const float*, double*,
                                                      cudaStream_t);

cudaError_t launch_assemble_dense(const Dims& d, const double* K0, const double* x,
                                  const double* Ae, const uint8_t* fixed, double* A,
                                  cudaStream_t st, long long ld, const double* w,
                                  const double* zll, const double* g, const double* Dinv) {
  const long long n = d.dofs();
  const long long na = w ? n + 1 : n;
  if (ld <= 0) ld = na;
  if (d.dim == 2)
    topo::launch(k_assemble_dense<2>, blocks_for(na * na), kThreads, 0, st, d, K0, x, Ae, fixed, A, ld, w,
                                                                  zll, g, Dinv);
  else
    topo::launch(k_assemble_dense<3>, blocks_for(na * na), kThreads, 0, st, d, K0, x, Ae, fixed, A, ld, w,
                                                                  zll, g, Dinv);
  return cudaGetLastError();
}

cudaError_t prepare_coarse_kernels(int n) {
  // the largest sizes, so that solvers of other sizes keep working
  (void)n;
  cudaError_t e =
      cudaFuncSetAttribute(k_cholesky_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_chol_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              200 * 1024);
}

// Newton-Schulz products (n <= kGjMaxN) or the block Gauss-Jordan workspace: W, the original
// diagonal, the row of Z tiles and P.
size_t coarse_scratch_doubles(int n) {
  if (n <= kGjMaxN) return 2 * (size_t)n * n;
  const size_t npad = ((size_t)n + kBg - 1) / kBg * kBg;
  return npad * npad + npad + (size_t)kBg * npad + (size_t)kBg * kBg;
}

cudaError_t launch_cholesky_inverse(int n, double* A, double* Ainv, int* info, cudaStream_t st,
                                    double* scratch, int* ns_bad, bool allow_ns) {
  if (n > kGjMaxN && scratch) {  // block Gauss-Jordan over many blocks
    const int npad = (n + kBg - 1) / kBg * kBg, nb = npad / kBg;
    double* W = scratch;
    double* a0 = W + (size_t)npad * npad;
    double* Z = a0 + npad;
    double* P = Z + (size_t)kBg * npad;
    topo::launch(k_bgj_setup, blocks_for((long long)npad * npad), kThreads, 0, st, n, npad,
                 (const double*)A, W, a0, info);
    for (int K = 0; K < nb; ++K) {
      topo::launch(k_bgj_pivot, 1, kBg * 8, 0, st, npad, K, (const double*)W, (const double*)a0,
                   P, info);
      topo::launch(k_bgj_zrow, nb, kBg * 8, 0, st, npad, K, (const double*)W, (const double*)P, Z,
                   (const int*)info);
      topo::launch(k_bgj_update, dim3(nb, nb), kBg * 8, 0, st, npad, K, W, (const double*)Z,
                   (const int*)info);
      topo::launch(k_bgj_final, nb, kBg * 8, 0, st, npad, K, W, (const double*)P,
                   (const double*)Z, (const int*)info);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    topo::launch(k_bgj_copy, blocks_for((long long)n * n), kThreads, 0, st, n, npad,
                 (const double*)W, Ainv, (const int*)info);
    return cudaGetLastError();
  }
  const int* only_if = nullptr;
  if (allow_ns && n <= kGjMaxN && scratch && ns_bad) {
    // X ping-pongs between Ainv and T so that the last product lands in Ainv (kNsSteps even)
    static_assert(kNsSteps % 2 == 0, "Newton-Schulz ping-pong ends in Ainv");
    double* R = scratch;
    double* T = scratch + (size_t)n * n;
    switch ((n + kGjRows - 1) / kGjRows) {
#define TOPO_GJ_CASE(E)                                                                            \
  case E:                                                                                          \
    topo::launch(k_gj32_start<E>, 1, kGjLanes * kGjRows, 0, st, n, (const double*)A, Ainv, info,  \
                 ns_bad);                                                                          \
    break;
      TOPO_GJ_CASE(1)
      TOPO_GJ_CASE(2)
      TOPO_GJ_CASE(3)
      TOPO_GJ_CASE(4)
      TOPO_GJ_CASE(5)
      TOPO_GJ_CASE(6)
      TOPO_GJ_CASE(7)
      default:
        topo::launch(k_gj32_start<8>, 1, kGjLanes * kGjRows, 0, st, n, (const double*)A, Ainv,
                     info, ns_bad);
#undef TOPO_GJ_CASE
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double* X = Ainv;
    double* Xn = T;
    for (int it = 0; it < kNsSteps; ++it) {
      const int last = (it == kNsSteps - 1) ? 1 : 0;
      const dim3 tiles((n + kNsTile - 1) / kNsTile, (n + kNsTile - 1) / kNsTile);
      topo::launch(k_ns_gemm, tiles, kNsTile * kNsTile, 0, st, n, (const double*)A,
                   (const double*)X, R, 2.0, -1.0, last, ns_bad);
      topo::launch(k_ns_gemm, tiles, kNsTile * kNsTile, 0, st, n, (const double*)X,
                   (const double*)R, Xn, 0.0, 1.0, 0, ns_bad);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      double* t = X;
      X = Xn;
      Xn = t;
    }
    only_if = ns_bad;  // the Cholesky kernels below run only if the check failed
  }
  const size_t smem = (size_t)n * n * sizeof(double);
  // row 0 of Ainv holds the original diagonal until the inverse overwrites it
  if (smem <= 200 * 1024)
    topo::launch(k_cholesky_smem, 1, 1024, smem, st, n, A, Ainv, info, only_if);
  else
    topo::launch(k_cholesky, 1, 1024, 0, st, n, A, Ainv, info, only_if);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int wpb = inv_warps(n);
  const size_t wsm = (size_t)wpb * n * sizeof(double);
  topo::launch(k_chol_inverse, (n + wpb - 1) / wpb, wpb * 32, wsm, st, n, A, Ainv, info, only_if);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dense_solve(int n, const double* Ainv, const float2* AinvDF, const T* b, T* z,
                               int nrhs, const CgScalars* sc, cudaStream_t st) {
  if (sizeof(T) == 4 && !AinvDF) return cudaErrorInvalidValue;
  dim3 grid(blocks_for((long long)n * 32), nrhs);
  topo::launch(k_dense_solve<T>, grid, kThreads, 0, st, n, Ainv, AinvDF, b, z, sc);
  return cudaGetLastError();
}
template cudaError_t launch_dense_solve<double>(int, const double*, const float2*, const double*,
                                                double*, int, const CgScalars*, cudaStream_t);
template cudaError_t launch_dense_solve<float>(int, const double*, const float2*, const float*,
                                               float*, int, const CgScalars*, cudaStream_t);

}  // namespace topo
