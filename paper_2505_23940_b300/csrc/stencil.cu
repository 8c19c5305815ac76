// Stencil kernels of the fractional-step time step (§2.3.1 of the paper):
//   predictor   u* of Eq. (4) with the direct-forcing blend of Eq. (5) fused,
//               RK stage combination fused, boundary faces set in the same pass
//   outflow     flux-balance scale of the zero-gradient outflow face
//   divergence  right-hand side D[(1 - eps) u* + eps u_c] of Eq. (9)
//   correct     u^{n+1} = u* - G phi of Eq. (10)
//   diagnostics max |u|, max |D u| and kinetic energy (FP64 reductions)
//
// Memory layout: every component dense, x fastest.  One thread per output
// face / cell; consecutive threads take consecutive x so every load and store
// of a warp is one or two 128-byte segments.
#include <cuda_runtime.h>

#include <cmath>

#include "fs_internal.cuh"

namespace fs {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(long long n, int threads = kThreads) {
  long long b = (n + threads - 1) / threads;
  return (int)(b > 0 ? b : 1);
}

template <typename T>
struct PredArgs {
  Geom<T> g;
  const T* uin[3];
  const T* un;
  T* out;
  T dt, a, b;
  int conv;
  const uint8_t* flags;
  T* num;
  T* den;
  T* fout;
  const double* body;
  double omega, cx, cy;
  const double* xf;
  const double* yf;
  const double* oscale;
};

// R(u) of Eq. (4) on the C-face (i, j, k): -div(u u) + nu lap(u) + body force.
// Same flux construction as the oracle (fluid.momentum_rhs), evaluated for one face.
template <typename T, int C>
__device__ __forceinline__ T momentum_rhs(const Geom<T>& g, const T* const* u, int conv, int i, int j, int k) {
  const int idx[3] = {i, j, k};
  T cv = T(0), df = T(0);
  // d == C: fluxes at the cell centres east (cell f) and west (cell f-1) of the face
  {
    int lo[3] = {i, j, k}, hi[3] = {i, j, k};
    lo[C] -= 1;
    hi[C] += 1;
    const T uW = ldv(g, u[C], C, lo[0], lo[1], lo[2]);
    const T u0 = ldv(g, u[C], C, i, j, k);
    const T uE = ldv(g, u[C], C, hi[0], hi[1], hi[2]);
    const T TE = T(0.5) * (u0 + uE), TW = T(0.5) * (uW + u0);
    T QE, QW;
    if (conv == FS_UPWIND1) {
      QE = TE > T(0) ? u0 : uE;
      QW = TW > T(0) ? uW : u0;
    } else {
      QE = TE;
      QW = TW;
    }
    T ihf, ihE, ihW;
    if (C == 1) {
      ihf = g.ihfy[j];
      ihE = g.ihy[j < g.ny ? j : g.ny - 1];
      ihW = g.ihy[j > 0 ? j - 1 : (g.per[1] ? g.ny - 1 : 0)];
    } else {
      ihf = ihE = ihW = (C == 0) ? g.ihx : g.ihz;
    }
    cv += (TE * QE - TW * QW) * ihf;
    df += ((uE - u0) * ihE - (u0 - uW) * ihW) * ihf;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d == C || d >= g.dim) continue;
    const T thc = (C == 1) ? g.thy[j] : T(0.5);
    int p_cd[3] = {i, j, k}, p_d[3] = {i, j, k}, p_c[3] = {i, j, k}, p_dm[3] = {i, j, k};
    p_cd[C] -= 1;
    p_cd[d] += 1;  // c-cell f-1, d-face m+1
    p_d[d] += 1;   // c-cell f,   d-face m+1
    p_c[C] -= 1;   // c-cell f-1, d-face m
    p_dm[d] -= 1;  // C component at d-cell m-1
    const T TN = (T(1) - thc) * ldv(g, u[d], d, p_cd[0], p_cd[1], p_cd[2]) + thc * ldv(g, u[d], d, p_d[0], p_d[1], p_d[2]);
    const T TS = (T(1) - thc) * ldv(g, u[d], d, p_c[0], p_c[1], p_c[2]) + thc * ldv(g, u[d], d, i, j, k);
    const T uS = ldv(g, u[C], C, p_dm[0], p_dm[1], p_dm[2]);
    const T u0 = ldv(g, u[C], C, i, j, k);
    const T uN = ldv(g, u[C], C, p_d[0], p_d[1], p_d[2]);
    const int m = idx[d];
    T thN, thS, ihd, ihfN, ihfS;
    if (d == 1) {
      thN = g.thy[m + 1];
      thS = g.thy[m];
      ihd = g.ihy[m];
      ihfN = g.ihfy[m + 1];
      ihfS = g.ihfy[m];
    } else {
      thN = thS = T(0.5);
      ihd = ihfN = ihfS = (d == 0) ? g.ihx : g.ihz;
    }
    T QN, QS;
    if (conv == FS_UPWIND1) {
      QN = TN > T(0) ? u0 : uN;
      QS = TS > T(0) ? uS : u0;
    } else {
      QN = (T(1) - thN) * u0 + thN * uN;
      QS = (T(1) - thS) * uS + thS * u0;
    }
    cv += (TN * QN - TS * QS) * ihd;
    df += ((uN - u0) * ihfN - (u0 - uS) * ihfS) * ihd;
  }
  T R = -cv + g.nu * df;
  if (C == 0 && g.bforce) R += g.bforce[j];
  return R;
}

// Rigid velocity V + omega x (r - r_c) at face position (px, py) (Eq. 23, solid points).
__device__ __forceinline__ void rigid_velocity(const double* body, double omega, double cx, double cy,
                                               double px, double py, double& vx, double& vy) {
  const double wx = body[0], wy = body[1];
  vx = body[2] - omega * (py - (cy + wy));
  vy = body[3] + omega * (px - (cx + wx));
}

template <typename T, int C>
__global__ void __launch_bounds__(kThreads) predictor_kernel(const PredArgs<T> A) {
  const Geom<T>& g = A.g;
  const int ex = g.ext(C, 0), ey = g.ext(C, 1), ez = g.ext(C, 2);
  const long long total = (long long)ex * ey * ez;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % ex);
    const long long r = t / ex;
    const int j = (int)(r % ey);
    const int k = (int)(r / ey);
    const int idx[3] = {i, j, k};
    const int ec = (C == 0) ? ex : (C == 1 ? ey : ez);
    T res;
    T fval = T(0);
    if (!g.per[C] && (idx[C] == 0 || idx[C] == ec - 1)) {
      // boundary face of a non-periodic direction: imposed normal velocity
      const int side = idx[C] == 0 ? 0 : 1;
      const int kind = g.bc[C][side];
      if (kind == FS_BC_OUTFLOW) {
        // u*[n] = s u[n-1], s from the flux balance (outflow_scale_kernel)
        res = T(*A.oscale) * A.uin[C][t - 1];
      } else if (kind == FS_BC_INFLOW) {
        res = g.bcv[C][side][C];
      } else {
        res = T(0);
      }
    } else {
      const T R = momentum_rhs<T, C>(g, A.uin, A.conv, i, j, k);
      const T u0 = A.uin[C][t];
      T v = u0 + A.dt * R;
      if (A.flags) {
        const uint8_t fl = A.flags[t];
        if (fl) {
          double px, py;
          if (C == 0) {
            px = A.xf[i];
            py = 0.5 * (A.yf[j] + A.yf[j + 1]);
          } else {
            px = 0.5 * (A.xf[i] + A.xf[i + 1]);
            py = A.yf[j];
          }
          double vx, vy;
          rigid_velocity(A.body, A.omega, A.cx, A.cy, px, py, vx, vy);
          T ut = T(C == 0 ? vx : vy);
          if (fl & 2) {
            const T dn = A.den[t];
            if (dn > T(0)) ut = A.num[t] / dn;
            A.num[t] = T(0);
            A.den[t] = T(0);
          }
          fval = -R + (ut - u0) / A.dt;   // Eq. (5) with eps = 1
          v = ut;                          // u* = u + dt (R + f) = u_s on forced faces
        }
      }
      res = (A.a != T(0)) ? A.a * A.un[t] + A.b * v : A.b * v;
    }
    A.out[t] = res;
    if (A.fout) A.fout[t] = fval;
  }
}

template <typename T>
__global__ void outflow_scale_kernel(const T* __restrict__ u0, int ex, int ny, int nz, const double* __restrict__ hy,
                                     double hz, double q_in, double* scale) {
  __shared__ double sh[kThreads];
  double s = 0.0;
  for (int t = threadIdx.x; t < ny * nz; t += blockDim.x) {
    const int j = t % ny, k = t / ny;
    s += (double)u0[(ex - 2) + (size_t)ex * (j + (size_t)ny * k)] * hy[j] * hz;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *scale = q_in / sh[0];
}

template <typename T>
struct DivArgs {
  Geom<T> g;
  const T* u[3];
  T* out;
  const uint8_t* flags[2];
  const double* body;
  double omega, cx, cy;
  const double* xf;
  const double* yf;
};

template <typename T>
__device__ __forceinline__ T blended(const DivArgs<T>& A, int c, size_t t, int i, int j) {
  if (A.flags[0] && c < 2 && A.flags[c][t]) {
    double px, py, vx, vy;
    if (c == 0) {
      px = A.xf[i];
      py = 0.5 * (A.yf[j] + A.yf[j + 1]);
    } else {
      px = 0.5 * (A.xf[i] + A.xf[i + 1]);
      py = A.yf[j];
    }
    rigid_velocity(A.body, A.omega, A.cx, A.cy, px, py, vx, vy);
    return T(c == 0 ? vx : vy);   // u_c on forced faces (Eq. 9)
  }
  return A.u[c][t];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) divergence_kernel(const DivArgs<T> A) {
  const Geom<T>& g = A.g;
  const long long total = (long long)g.nx * g.ny * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const long long r = t / g.nx;
    const int j = (int)(r % g.ny);
    const int k = (int)(r / g.ny);
    T s = T(0);
    {
      const int ex = g.ext(0, 0);
      const size_t base = (size_t)ex * (j + (size_t)g.ny * k);
      const int ip = (i + 1 < ex) ? i + 1 : 0;
      s += (blended(A, 0, base + ip, ip, j) - blended(A, 0, base + i, i, j)) * g.ihx;
    }
    {
      const int ey = g.ext(1, 1);
      const int jp = (j + 1 < ey) ? j + 1 : 0;
      const size_t b0 = i + (size_t)g.nx * ((size_t)ey * k);
      s += (blended(A, 1, b0 + (size_t)g.nx * jp, i, jp) - blended(A, 1, b0 + (size_t)g.nx * j, i, j)) * g.ihy[j];
    }
    if (g.dim == 3) {
      const int ez = g.ext(2, 2);
      const int kp = (k + 1 < ez) ? k + 1 : 0;
      const size_t b0 = i + (size_t)g.nx * j;
      const size_t pl = (size_t)g.nx * g.ny;
      s += (A.u[2][b0 + pl * kp] - A.u[2][b0 + pl * k]) * g.ihz;
    }
    A.out[t] = s;
  }
}

template <typename T, int C>
__global__ void __launch_bounds__(kThreads) correct_kernel(const Geom<T> g, const T* __restrict__ us,
                                                           const T* __restrict__ phi, T* __restrict__ un) {
  const int ex = g.ext(C, 0), ey = g.ext(C, 1), ez = g.ext(C, 2);
  const long long total = (long long)ex * ey * ez;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % ex);
    const long long r = t / ex;
    const int j = (int)(r % ey);
    const int k = (int)(r / ey);
    int idx[3] = {i, j, k};
    const int ec = (C == 0) ? ex : (C == 1 ? ey : ez);
    T v = us[t];
    if (g.per[C] || (idx[C] > 0 && idx[C] < ec - 1)) {
      // G phi at the face: (phi[cell f] - phi[cell f-1]) / hf
      int lo[3] = {i, j, k};
      const int nC = (C == 0) ? g.nx : (C == 1 ? g.ny : g.nz);
      lo[C] = idx[C] > 0 ? idx[C] - 1 : nC - 1;
      const size_t c0 = idx[0] + (size_t)g.nx * (idx[1] + (size_t)g.ny * idx[2]);
      const size_t c1 = lo[0] + (size_t)g.nx * (lo[1] + (size_t)g.ny * lo[2]);
      const T ihf = (C == 0) ? g.ihx : (C == 1 ? g.ihfy[j] : g.ihz);
      v -= (phi[c0] - phi[c1]) * ihf;
    }
    un[t] = v;
  }
}

template <typename T>
__global__ void to_pressure_kernel(const T* __restrict__ phi, double* __restrict__ p, long long n, double scale) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    p[t] = (double)phi[t] * scale;
}

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // v >= 0: the IEEE bit pattern orders like the integer
  atomicMax((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}

// out[0] = max |u|, out[1] = max |D u|, out[2] = kinetic energy (atomics; FP64)
template <typename T>
__global__ void diag_faces_kernel(const Geom<T> g, const T* __restrict__ u, int c, const double* __restrict__ hy,
                                  const double* __restrict__ hfy, double* out) {
  __shared__ double smax[kThreads], ske[kThreads];
  const int ex = g.ext(c, 0), ey = g.ext(c, 1), ez = g.ext(c, 2);
  const long long total = (long long)ex * ey * ez;
  double m = 0.0, ke = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % ex);
    const long long r = t / ex;
    const int j = (int)(r % ey);
    (void)i;
    const double v = (double)u[t];
    m = fmax(m, fabs(v));
    // face control volume: hf along c times the cell widths across
    const double hz = g.dim == 3 ? (double)g.hz : 1.0;
    double vol;
    if (c == 0) vol = (double)g.hx * hy[j] * hz;
    else if (c == 1) vol = (double)g.hx * hfy[j] * hz;
    else vol = (double)g.hx * hy[j] * hz;
    ke += 0.5 * v * v * vol;
  }
  smax[threadIdx.x] = m;
  ske[threadIdx.x] = ke;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
      ske[threadIdx.x] += ske[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomic_max_pos(&out[0], smax[0]);
    atomicAdd(&out[2], ske[0]);
  }
}

template <typename T>
__global__ void diag_div_kernel(const Geom<T> g, const T* __restrict__ u0, const T* __restrict__ u1,
                                const T* __restrict__ u2, const double* __restrict__ hy, double* out) {
  __shared__ double smax[kThreads];
  const long long total = (long long)g.nx * g.ny * g.nz;
  double m = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const long long r = t / g.nx;
    const int j = (int)(r % g.ny);
    const int k = (int)(r / g.ny);
    const int ex = g.ext(0, 0), ey = g.ext(1, 1), ez = g.ext(2, 2);
    const int ip = (i + 1 < ex) ? i + 1 : 0, jp = (j + 1 < ey) ? j + 1 : 0, kp = (k + 1 < ez) ? k + 1 : 0;
    double s = ((double)u0[ip + (size_t)ex * (j + (size_t)g.ny * k)] - (double)u0[i + (size_t)ex * (j + (size_t)g.ny * k)]) / g.hx;
    s += ((double)u1[i + (size_t)g.nx * (jp + (size_t)ey * k)] - (double)u1[i + (size_t)g.nx * (j + (size_t)ey * k)]) / hy[j];
    if (g.dim == 3)
      s += ((double)u2[i + (size_t)g.nx * (j + (size_t)g.ny * kp)] - (double)u2[i + (size_t)g.nx * (j + (size_t)g.ny * k)]) / g.hz;
    m = fmax(m, fabs(s));
  }
  smax[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomic_max_pos(&out[1], smax[0]);
}

int grid_blocks(long long n) {
  int b = blocks_for(n);
  // enough CTAs for every SM several times over; grid-stride loops cover the rest
  const int cap = 148 * 16;
  return b < cap ? b : cap;
}

}  // namespace

template <typename T>
void launch_predictor(fs_grid* G, T* const* uin, T* const* un, T* const* out, double dt, double a, double b,
                      const double* body_state) {
  PredArgs<T> A;
  A.g = G->geom<T>();
  for (int c = 0; c < 3; ++c) A.uin[c] = c < G->dim ? uin[c] : nullptr;
  A.dt = (T)dt;
  A.a = (T)a;
  A.b = (T)b;
  A.conv = G->conv;
  A.body = body_state;
  A.omega = G->ib.omega;
  A.cx = G->ib.centre[0];
  A.cy = G->ib.centre[1];
  A.xf = G->xf64[0];
  A.yf = G->xf64[1];
  A.oscale = G->scal;
  for (int c = 0; c < G->dim; ++c) {
    A.un = un ? un[c] : nullptr;
    A.out = out[c];
    const bool ibc = G->has_body && c < 2;
    A.flags = ibc ? G->ib.flags[c] : nullptr;
    A.num = ibc ? (T*)G->ib.num[c] : nullptr;
    A.den = ibc ? (T*)G->ib.den[c] : nullptr;
    A.fout = ibc ? (T*)G->ib.f[c] : nullptr;
    const long long n = (long long)A.g.ext(c, 0) * A.g.ext(c, 1) * A.g.ext(c, 2);
    const int nb = grid_blocks(n);
    if (c == 0) FS_LAUNCH(G, "predictor_u", predictor_kernel<T, 0><<<nb, kThreads, 0, G->stream>>>(A));
    else if (c == 1) FS_LAUNCH(G, "predictor_v", predictor_kernel<T, 1><<<nb, kThreads, 0, G->stream>>>(A));
    else FS_LAUNCH(G, "predictor_w", predictor_kernel<T, 2><<<nb, kThreads, 0, G->stream>>>(A));
  }
}

template <typename T>
void launch_outflow_flux(fs_grid* G, T* const* uin) {
  if (G->per[0] || G->bc[0][1] != FS_BC_OUTFLOW) return;
  double q_in = 0.0;
  if (G->bc[0][0] == FS_BC_INFLOW) {
    double area = 0.0;
    for (int j = 0; j < G->ny; ++j) area += G->h[1][j];
    area *= (G->dim == 3 ? G->hz * G->nz : 1.0);
    q_in = G->bcv[0][0][0] * area;
  }
  FS_LAUNCH(G, "outflow_scale", outflow_scale_kernel<T><<<1, kThreads, 0, G->stream>>>(uin[0], G->nx + 1, G->ny, G->nz, G->hy64,
                                                         G->dim == 3 ? G->hz : 1.0, q_in, G->scal));
}

template <typename T>
void launch_divergence(fs_grid* G, T* const* u, T* out, const double* body_state) {
  DivArgs<T> A;
  A.g = G->geom<T>();
  for (int c = 0; c < 3; ++c) A.u[c] = c < G->dim ? u[c] : nullptr;
  A.out = out;
  A.flags[0] = G->has_body ? G->ib.flags[0] : nullptr;
  A.flags[1] = G->has_body ? G->ib.flags[1] : nullptr;
  A.body = body_state;
  A.omega = G->ib.omega;
  A.cx = G->ib.centre[0];
  A.cy = G->ib.centre[1];
  A.xf = G->xf64[0];
  A.yf = G->xf64[1];
  FS_LAUNCH(G, "divergence", divergence_kernel<T><<<grid_blocks((long long)G->nx * G->ny * G->nz), kThreads, 0, G->stream>>>(A));
}

template <typename T>
void launch_correct(fs_grid* G, T* const* ustar, const T* phi, T* const* unew) {
  const Geom<T> g = G->geom<T>();
  for (int c = 0; c < G->dim; ++c) {
    const long long n = (long long)g.ext(c, 0) * g.ext(c, 1) * g.ext(c, 2);
    const int nb = grid_blocks(n);
    if (c == 0) FS_LAUNCH(G, "correct_u", correct_kernel<T, 0><<<nb, kThreads, 0, G->stream>>>(g, ustar[0], phi, unew[0]));
    else if (c == 1) FS_LAUNCH(G, "correct_v", correct_kernel<T, 1><<<nb, kThreads, 0, G->stream>>>(g, ustar[1], phi, unew[1]));
    else FS_LAUNCH(G, "correct_w", correct_kernel<T, 2><<<nb, kThreads, 0, G->stream>>>(g, ustar[2], phi, unew[2]));
  }
}

template <typename T>
void launch_to_pressure(fs_grid* G, const T* phi, double* p, double scale) {
  const long long n = (long long)G->nx * G->ny * G->nz;
  FS_LAUNCH(G, "to_pressure", to_pressure_kernel<T><<<grid_blocks(n), kThreads, 0, G->stream>>>(phi, p, n, scale));
}

template <typename T>
void launch_diagnostics(fs_grid* G, T* const* u, double* out3) {
  const Geom<T> g = G->geom<T>();
  cudaMemsetAsync(out3, 0, 3 * sizeof(double), G->stream);
  double* hfy = G->hfy64;
  for (int c = 0; c < G->dim; ++c) {
    const long long n = (long long)g.ext(c, 0) * g.ext(c, 1) * g.ext(c, 2);
    FS_LAUNCH(G, "diag_faces", diag_faces_kernel<T><<<grid_blocks(n), kThreads, 0, G->stream>>>(g, u[c], c, G->hy64, hfy, out3));
  }
  FS_LAUNCH(G, "diag_div", diag_div_kernel<T><<<grid_blocks((long long)G->nx * G->ny * G->nz), kThreads, 0, G->stream>>>(
      g, u[0], u[1], G->dim == 3 ? u[2] : u[1], G->hy64, out3));
}

#define FS_INST(T)                                                                                                 \
  template void launch_predictor<T>(fs_grid*, T* const*, T* const*, T* const*, double, double, double,          \
                                    const double*);                                                              \
  template void launch_outflow_flux<T>(fs_grid*, T* const*);                                                     \
  template void launch_divergence<T>(fs_grid*, T* const*, T*, const double*);                                    \
  template void launch_correct<T>(fs_grid*, T* const*, const T*, T* const*);                                     \
  template void launch_to_pressure<T>(fs_grid*, const T*, double*, double);                                      \
  template void launch_diagnostics<T>(fs_grid*, T* const*, double*);
FS_INST(float)
FS_INST(double)
#undef FS_INST

}  // namespace fs
