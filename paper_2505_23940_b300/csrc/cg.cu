// Conjugate-gradient solve of the pressure Poisson equation D G p = b (Eq. 9)
// with the Krylov iteration the paper uses (§2.5, Table 1: CG by default),
// fs_solve_pressure_cg.  It reaches the same zero-mean solution as the direct
// transform solver of poisson.cu and serves as its cross-check and as the
// solver form the paper states.
//
// L = D G is symmetric in the cell-volume inner product, so CG runs on
//   A x = r,  A = -V L (symmetric positive semi-definite),  r = -V b,
// with the right-hand side's plain mean removed (the constant null space of a
// grid without Dirichlet pressure), optional Jacobi preconditioning by diag(A),
// and the result shifted to zero volume-weighted mean.  Everything is FP64.
// The scalars of the iteration stay on the device: each kernel reads the dot
// products the previous one accumulated, so an iteration is three launches
// with no host round trip; the host reads the residual every few iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fs_internal.cuh"

namespace fs {

namespace {

constexpr int kCgT = 256;

// slots of the device scalar array
enum { S_RZ = 0, S_PQ = 1, S_RZN = 2, S_RR = 3, S_VX = 4, S_RR0 = 6, S_SUM = 7, S_N = 8 };

struct CgGeom {
  int dim, nx, ny, nz;
  int per[3];
  double ihx, ihz, hx, hz;
  const double* ihy;    // 1 / h_y  (ny)
  const double* ihfy;   // 1 / hf_y (ny + 1)
  const double* hy;     // h_y      (ny)
  int jacobi;
};

__device__ __forceinline__ double cell_volume(const CgGeom& g, int j) {
  return g.hx * g.hy[j] * (g.dim == 3 ? g.hz : 1.0);
}

// (A x)(c) = V(c) sum_d (G_lo - G_hi) / h_d(c), G the face gradient, 0 on the
// faces of non-periodic boundaries (G p . n = 0).
__device__ __forceinline__ double apply_A(const CgGeom& g, const double* __restrict__ x, int i, int j, int k) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const size_t plane = (size_t)nx * ny;
  const size_t c = i + (size_t)nx * j + plane * k;
  const double xc = x[c];
  double s = 0.0;
  {
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    double t = 0.0;
    if (g.per[0] || i > 0) t += (xc - x[c - i + im]) * g.ihx;
    if (g.per[0] || i < nx - 1) t -= (x[c - i + ip] - xc) * g.ihx;
    s += t * g.ihx;
  }
  {
    const int jm = j > 0 ? j - 1 : ny - 1, jp = j < ny - 1 ? j + 1 : 0;
    double t = 0.0;
    if (g.per[1] || j > 0) t += (xc - x[i + (size_t)nx * jm + plane * k]) * g.ihfy[j];
    if (g.per[1] || j < ny - 1) t -= (x[i + (size_t)nx * jp + plane * k] - xc) * g.ihfy[j + 1];
    s += t * g.ihy[j];
  }
  if (g.dim == 3) {
    const int km = k > 0 ? k - 1 : nz - 1, kp = k < nz - 1 ? k + 1 : 0;
    double t = 0.0;
    if (g.per[2] || k > 0) t += (xc - x[i + (size_t)nx * j + plane * km]) * g.ihz;
    if (g.per[2] || k < nz - 1) t -= (x[i + (size_t)nx * j + plane * kp] - xc) * g.ihz;
    s += t * g.ihz;
  }
  return cell_volume(g, j) * s;
}

// diag(A) at cell (i, j, k) from the metrics alone.
__device__ __forceinline__ double diag_A(const CgGeom& g, int i, int j, int k) {
  double dg = 0.0;
  dg += ((g.per[0] || i > 0) + (g.per[0] || i < g.nx - 1)) * g.ihx * g.ihx;
  dg += (((g.per[1] || j > 0) ? g.ihfy[j] : 0.0) + ((g.per[1] || j < g.ny - 1) ? g.ihfy[j + 1] : 0.0)) * g.ihy[j];
  if (g.dim == 3) dg += ((g.per[2] || k > 0) + (g.per[2] || k < g.nz - 1)) * g.ihz * g.ihz;
  return cell_volume(g, j) * dg;
}

// Block sum of up to two values, one FP64 atomic per block and value.
__device__ __forceinline__ void block_add(double a, double b, double* sa, double* sb) {
  __shared__ double ra[kCgT / 32], rb[kCgT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) {
    ra[w] = a;
    rb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) {
      ta += ra[q];
      tb += rb[q];
    }
    if (sa) atomicAdd(sa, ta);
    if (sb) atomicAdd(sb, tb);
  }
}

// grid-stride loop over cells; (i, j, k) from the linear index
#define CG_CELLS(g, c, i, j, k)                                                                     \
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x, n_ = (size_t)g.nx * g.ny * g.nz; c < n_; \
       c += (size_t)gridDim.x * blockDim.x)                                                          \
    if (const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((size_t)g.nx * g.ny)); true)

__global__ void __launch_bounds__(kCgT) cg_init_kernel(const CgGeom g, const double* __restrict__ b,
                                                       double* __restrict__ r, double* __restrict__ x, double* S) {
  double sum = 0.0;
  CG_CELLS(g, c, i, j, k) {
    (void)i;
    (void)k;
    const double v = -cell_volume(g, j) * b[c];
    r[c] = v;
    x[c] = 0.0;
    sum += v;
  }
  block_add(sum, 0.0, S + S_SUM, nullptr);
}

__global__ void __launch_bounds__(kCgT) cg_init2_kernel(const CgGeom g, double* __restrict__ r, double* z,
                                                        double* __restrict__ p, double* S) {
  const double mean = S[S_SUM] / ((double)g.nx * g.ny * g.nz);
  double rz = 0.0, rr = 0.0;
  CG_CELLS(g, c, i, j, k) {
    const double v = r[c] - mean;
    r[c] = v;
    double zi = v;
    if (g.jacobi) {
      zi = v / diag_A(g, i, j, k);
      z[c] = zi;
    }
    p[c] = zi;
    rz += v * zi;
    rr += v * v;
  }
  block_add(rz, rr, S + S_RZN, S + S_RR0);
}

// q = A p, pq += p . q; the first thread rotates rz and clears the update's sums.
__global__ void __launch_bounds__(kCgT) cg_apply_kernel(const CgGeom g, const double* __restrict__ p,
                                                        double* __restrict__ q, double* S) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S[S_RZ] = S[S_RZN];
    S[S_RZN] = 0.0;
    S[S_RR] = 0.0;
  }
  double pq = 0.0;
  CG_CELLS(g, c, i, j, k) {
    const double v = apply_A(g, p, i, j, k);
    q[c] = v;
    pq += p[c] * v;
  }
  block_add(pq, 0.0, S + S_PQ, nullptr);
}

// alpha = rz / pq; x += alpha p; r -= alpha q; z = M^-1 r; rz_new, rr accumulated.
__global__ void __launch_bounds__(kCgT) cg_update_kernel(const CgGeom g, const double* __restrict__ p,
                                                         const double* __restrict__ q, double* __restrict__ x,
                                                         double* __restrict__ r, double* z, double* S) {
  const double alpha = S[S_RZ] / S[S_PQ];
  double rz = 0.0, rr = 0.0;
  CG_CELLS(g, c, i, j, k) {
    x[c] += alpha * p[c];
    const double v = r[c] - alpha * q[c];
    r[c] = v;
    double zi = v;
    if (g.jacobi) {
      zi = v / diag_A(g, i, j, k);
      z[c] = zi;
    }
    rz += v * zi;
    rr += v * v;
  }
  block_add(rz, rr, S + S_RZN, S + S_RR);
}

// beta = rz_new / rz; p = z + beta p; the first thread clears pq for the next apply.
__global__ void __launch_bounds__(kCgT) cg_dir_kernel(const CgGeom g, const double* z,
                                                      double* __restrict__ p, double* S) {
  const double beta = S[S_RZN] / S[S_RZ];
  if (blockIdx.x == 0 && threadIdx.x == 0) S[S_PQ] = 0.0;
  CG_CELLS(g, c, i, j, k) {
    (void)i;
    (void)j;
    (void)k;
    p[c] = z[c] + beta * p[c];
  }
}

__global__ void __launch_bounds__(kCgT) cg_vsum_kernel(const CgGeom g, const double* __restrict__ x, double* S) {
  double s = 0.0;
  CG_CELLS(g, c, i, j, k) {
    (void)i;
    (void)k;
    s += cell_volume(g, j) * x[c];
  }
  block_add(s, 0.0, S + S_VX, nullptr);
}

__global__ void __launch_bounds__(kCgT) cg_shift_kernel(const CgGeom g, double* __restrict__ x, const double* S,
                                                        double vtot) {
  const double m = S[S_VX] / vtot;
  CG_CELLS(g, c, i, j, k) {
    (void)i;
    (void)j;
    (void)k;
    x[c] -= m;
  }
}

}  // namespace

}  // namespace fs

using namespace fs;

extern "C" int fs_solve_pressure_cg(fs_grid* G, const double* rhs, double* p, double tol, int maxit, int jacobi,
                                    int* iters, double* relres) {
  if (!G || !rhs || !p) return set_error(FS_ERR_ARG, "NULL argument");
  if (G->prec == FS_MIXED)
    return set_error(FS_ERR_UNSUPPORTED, "fs_solve_pressure_cg takes FP64 data; use an FS_FP64 grid");
  if (!(tol > 0.0) || maxit < 1) return set_error(FS_ERR_ARG, "fs_solve_pressure_cg: tol must be > 0, maxit >= 1");
  if (rhs == p) return set_error(FS_ERR_ARG, "fs_solve_pressure_cg: rhs and p must not alias");
  const size_t n = (size_t)G->nx * G->ny * G->nz;
  if (!G->cg) {
    if (cudaMalloc(&G->cg, (3 * n + 16) * sizeof(double)) != cudaSuccess)
      return set_error(FS_ERR_CUDA, "allocating conjugate-gradient workspace");
  }
  double* r = (double*)G->cg;
  double* q = r + n;
  double* d = q + n;               // search direction
  double* S = d + n;
  double* z = jacobi ? (double*)G->spec : r;   // preconditioned residual (spec holds n doubles)
  CgGeom g;
  g.dim = G->dim;
  g.nx = G->nx;
  g.ny = G->ny;
  g.nz = G->nz;
  for (int a = 0; a < 3; ++a) g.per[a] = G->per[a];
  g.hx = G->hx;
  g.hz = G->dim == 3 ? G->hz : 1.0;
  g.ihx = 1.0 / G->hx;
  g.ihz = 1.0 / g.hz;
  g.ihy = G->ihy64;
  g.ihfy = G->ihfy64;
  g.hy = G->hy64;
  g.jacobi = jacobi ? 1 : 0;
  double vtot = 0.0;
  for (int j = 0; j < G->ny; ++j) vtot += G->h[1][j];
  vtot *= G->hx * G->nx * (G->dim == 3 ? G->hz * G->nz : 1.0);
  const int blocks = (int)std::min<size_t>((n + kCgT - 1) / kCgT, 148 * 8);
  cudaStream_t s = G->stream;
  cudaMemsetAsync(S, 0, 16 * sizeof(double), s);
  FS_LAUNCH(G, "cg_init", cg_init_kernel<<<blocks, kCgT, 0, s>>>(g, rhs, r, p, S));
  FS_LAUNCH(G, "cg_init", cg_init2_kernel<<<blocks, kCgT, 0, s>>>(g, r, z, d, S));
  double host[8];
  cudaError_t e = cudaMemcpyAsync(host, S, 8 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "fs_solve_pressure_cg init");
  const double rr0 = host[S_RR0];
  int it = 0;
  double rel = 0.0;
  if (rr0 > 0.0) {
    constexpr int kCheck = 8;
    while (it < maxit) {
      FS_LAUNCH(G, "cg_apply", cg_apply_kernel<<<blocks, kCgT, 0, s>>>(g, d, q, S));
      FS_LAUNCH(G, "cg_update", cg_update_kernel<<<blocks, kCgT, 0, s>>>(g, d, q, p, r, z, S));
      ++it;
      if (it % kCheck == 0 || it == maxit) {
        e = cudaMemcpyAsync(host, S, 8 * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_check(e, "fs_solve_pressure_cg");
        rel = std::sqrt(host[S_RR] / rr0);
        if (!(rel == rel)) return set_error(FS_ERR_DIVERGED, "fs_solve_pressure_cg: NaN residual");
        if (rel <= tol) break;
      }
      FS_LAUNCH(G, "cg_dir", cg_dir_kernel<<<blocks, kCgT, 0, s>>>(g, z, d, S));
    }
  }
  FS_LAUNCH(G, "cg_gauge", cg_vsum_kernel<<<blocks, kCgT, 0, s>>>(g, p, S));
  FS_LAUNCH(G, "cg_gauge", cg_shift_kernel<<<blocks, kCgT, 0, s>>>(g, p, S, vtot));
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return cuda_check(cudaGetLastError(), "fs_solve_pressure_cg");
}
