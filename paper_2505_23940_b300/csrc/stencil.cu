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

#include <type_traits>

#include "fs_internal.cuh"
#include "tma.cuh"

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
  const T* un[3];
  T* out[3];
  T dt, a, b;
  int conv;
  int X, Y;                  // thread grid (largest component extents along x and y)
  int jlo;                   // first row of the vector kernels (walls: 2; the wall rows run apart)
  const uint8_t* flags[2];   // IB (2-D): per-face flags, accumulators and forcing output
  T* num[2];
  T* den[2];
  T* fout[2];
  const double* body;
  double omega, cx, cy;
  const double* xf;
  const double* yf;
  const double* oscale;
  T ihy0;                    // 1 / h_y of a uniform periodic y (predictor3_kernel<T, true>)
  const uint8_t* flags3[3];  // static 3-D body (boxes): per-face flags, forced faces take u_s = 0
  T* fout3[3];               // and the forcing term f on forced faces (zero from the start elsewhere)
  const T* nut[4];           // Smagorinsky eddy viscosity: cell centres, xy, xz, yz edges (or null)
};

// Velocity access around the face (i, j, k) with every boundary rule (ldv).
template <typename T>
struct AccGhost {
  const Geom<T>* g;
  const T* const* u;
  int i, j, k;
  __device__ __forceinline__ T operator()(int c, int di, int dj, int dk) const {
    return ldv(*g, u[c], c, i + di, j + dj, k + dk);
  }
};

// Velocity access for a face whose whole stencil lies inside: the wrapped
// neighbour indices are formed once per thread, every load is two 32-bit
// multiply-adds away (field sizes are checked below 2^31 at grid creation).
template <typename T>
struct AccFast {
  const T* const* u;
  int xo[3], yo[3], zo[3];   // neighbour index for offsets -1, 0, +1 (periodic wrap applied)
  int ex[3], exy[3];         // per component: x extent and plane size
  __device__ __forceinline__ AccFast(const Geom<T>& g, const T* const* uu, int i, int j, int k) : u(uu) {
    const int n[3] = {g.nx, g.ny, g.nz};
    const int p[3] = {i, j, k};
    int* o[3] = {xo, yo, zo};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      o[d][0] = p[d] - 1;
      o[d][1] = p[d];
      o[d][2] = p[d] + 1;
      if (g.per[d]) {
        if (p[d] == 0) o[d][0] = n[d] - 1;
        if (p[d] == n[d] - 1) o[d][2] = 0;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ex[c] = g.ext(c, 0);
      exy[c] = ex[c] * g.ext(c, 1);
    }
  }
  __device__ __forceinline__ T operator()(int c, int di, int dj, int dk) const {
    return __ldg(u[c] + (xo[di + 1] + ex[c] * yo[dj + 1] + exy[c] * zo[dk + 1]));
  }
};

// R(u) of Eq. (4) on the C-face (i, j, k): -div(u u) + nu lap(u) + body force.
// Same flux construction as the oracle (fluid.momentum_rhs), evaluated for one face.
template <typename T, int C, typename Acc>
__device__ __forceinline__ T momentum_rhs(const Geom<T>& g, const Acc& U, int conv, int i, int j, int k) {
  const int idx[3] = {i, j, k};
  T cv = T(0), df = T(0);
  // unit offsets along C
  constexpr int cx = C == 0, cy = C == 1, cz = C == 2;
  // d == C: fluxes at the cell centres east (cell f) and west (cell f-1) of the face
  {
    const T uW = U(C, -cx, -cy, -cz);
    const T u0 = U(C, 0, 0, 0);
    const T uE = U(C, cx, cy, cz);
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
    const int dx = d == 0, dy = d == 1, dz = d == 2;
    const T thc = (C == 1) ? g.thy[j] : T(0.5);
    // transport u_d at (c-cell f-1 | f, d-face m+1 | m); C component at d-cells m-1, m, m+1
    const T TN = (T(1) - thc) * U(d, dx - cx, dy - cy, dz - cz) + thc * U(d, dx, dy, dz);
    const T TS = (T(1) - thc) * U(d, -cx, -cy, -cz) + thc * U(d, 0, 0, 0);
    const T uS = U(C, -dx, -dy, -dz);
    const T u0 = U(C, 0, 0, 0);
    const T uN = U(C, dx, dy, dz);
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


// Predictor for the C-face (i, j, k): Eq. (4), the direct-forcing blend of
// Eq. (5) on forced faces, the RK stage combination, and the imposed normal
// velocity on boundary faces.
template <typename T, int C, typename Acc>
__device__ __forceinline__ void predict_face(const PredArgs<T>& A, const Acc& U, int i, int j, int k) {
  const Geom<T>& g = A.g;
  const int ex = g.ext(C, 0), ey = g.ext(C, 1), ez = g.ext(C, 2);
  if (i >= ex || j >= ey || k >= ez) return;
  const int t = i + ex * (j + ey * k);
  const int idx[3] = {i, j, k};
  const int ec = (C == 0) ? ex : (C == 1 ? ey : ez);
  T res;
  T fval = T(0);
  if (!g.per[C] && (idx[C] == 0 || idx[C] == ec - 1)) {
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
    const T R = momentum_rhs<T, C>(g, U, A.conv, i, j, k);
    const T u0 = A.uin[C][t];
    T v = u0 + A.dt * R;
    if (C < 2 && A.flags[0]) {
      const uint8_t fl = A.flags[C][t];
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
          const T dn = A.den[C][t];
          if (dn > T(0)) ut = A.num[C][t] / dn;
          A.num[C][t] = T(0);
          A.den[C][t] = T(0);
        }
        fval = -R + (ut - u0) / A.dt;   // Eq. (5) with eps = 1
        v = ut;                          // u* = u + dt (R + f) = u_s on forced faces
      }
    }
    if (A.flags3[0] && A.flags3[C][t]) {   // static 3-D body: u_s = 0
      fval = -R - u0 / A.dt;
      v = T(0);
    }
    res = (A.a != T(0)) ? A.a * A.un[C][t] + A.b * v : A.b * v;
  }
  A.out[C][t] = res;
  if (C < 2 && A.fout[0]) A.fout[C][t] = fval;
  if (A.fout3[0] && A.flags3[C][t]) A.fout3[C][t] = fval;   // off forced faces f stays 0 (static body)
}

// One thread per cell position (i, j, k) computes every component's face there.
template <typename T>
__global__ void __launch_bounds__(kThreads) predictor_kernel(const PredArgs<T> A) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= A.X || j >= A.Y) return;
  const Geom<T>& g = A.g;
  bool fast = true;
  if (!g.per[0]) fast = fast && i >= 2 && i <= g.nx - 2;
  if (!g.per[1]) fast = fast && j >= 2 && j <= g.ny - 2;
  if (g.dim == 3 && !g.per[2]) fast = fast && k >= 2 && k <= g.nz - 2;
  if (fast) {
    const AccFast<T> U(g, A.uin, i, j, k);
    predict_face<T, 0>(A, U, i, j, k);
    predict_face<T, 1>(A, U, i, j, k);
    if (g.dim == 3) predict_face<T, 2>(A, U, i, j, k);
  } else {
    const AccGhost<T> U{&g, A.uin, i, j, k};
    predict_face<T, 0>(A, U, i, j, k);
    predict_face<T, 1>(A, U, i, j, k);
    if (g.dim == 3) predict_face<T, 2>(A, U, i, j, k);
  }
}

// The 27 neighbour values of cell (i, j, k) that the three face updates of
// Eq. (4) need in the 3-D central scheme; names give the offsets in x, y, z
// (0, M = -1, P = +1).
template <typename T>
struct Nb27 {
  T u000, uM00, uP00, u0M0, u0P0, u00M, u00P, uPM0, uP0M;
  T v000, vM00, vP00, v0M0, v0P0, v00M, v00P, vMP0, v0PM;
  T w000, wM00, wP00, w0M0, w0P0, w00M, w00P, wM0P, w0MP;
};

// y metrics at row j: 1/h_y[j], 1/h_y[j-1], 1/hf_y[j], 1/hf_y[j+1], theta_y[j], theta_y[j+1]
template <typename T>
struct YMet {
  T ihyj, ihyjm, ihfj, ihfjp, thj, thjp;
};

template <typename T, bool YPER>
__device__ __forceinline__ YMet<T> ymet(const PredArgs<T>& A, int j) {
  YMet<T> m;
  if (YPER) {
    m.ihyj = m.ihyjm = m.ihfj = m.ihfjp = A.ihy0;
    m.thj = m.thjp = T(0.5);
  } else {
    const Geom<T>& g = A.g;
    m.ihyj = g.ihy[j];
    m.ihyjm = g.ihy[j - 1];
    m.ihfj = g.ihfy[j];
    m.ihfjp = g.ihfy[j + 1];
    m.thj = g.thy[j];
    m.thjp = g.thy[j + 1];
  }
  return m;
}

// R(u) of Eq. (4) on the x-, y- and z-faces of one cell, central convection;
// the arithmetic is that of momentum_rhs with the interior metrics.
template <typename T>
__device__ __forceinline__ void rhs3(const Nb27<T>& n, const YMet<T>& m, T ihx, T ihz, T nu, T bf, T& Ru, T& Rv,
                                     T& Rw) {
  const T h = T(0.5);
  {  // u on the x-face
    const T TE = h * (n.u000 + n.uP00), TW = h * (n.uM00 + n.u000);
    T cv = (TE * TE - TW * TW) * ihx;
    T df = ((n.uP00 - n.u000) * ihx - (n.u000 - n.uM00) * ihx) * ihx;
    const T TN = h * (n.vMP0 + n.v0P0), TS = h * (n.vM00 + n.v000);
    const T QN = (T(1) - m.thjp) * n.u000 + m.thjp * n.u0P0, QS = (T(1) - m.thj) * n.u0M0 + m.thj * n.u000;
    cv += (TN * QN - TS * QS) * m.ihyj;
    df += ((n.u0P0 - n.u000) * m.ihfjp - (n.u000 - n.u0M0) * m.ihfj) * m.ihyj;
    const T TT = h * (n.wM0P + n.w00P), TB = h * (n.wM00 + n.w000);
    const T QT = h * (n.u000 + n.u00P), QB = h * (n.u00M + n.u000);
    cv += (TT * QT - TB * QB) * ihz;
    df += ((n.u00P - n.u000) * ihz - (n.u000 - n.u00M) * ihz) * ihz;
    Ru = -cv + nu * df + bf;
  }
  {  // v on the y-face
    const T TE = h * (n.v000 + n.v0P0), TW = h * (n.v0M0 + n.v000);
    T cv = (TE * TE - TW * TW) * m.ihfj;
    T df = ((n.v0P0 - n.v000) * m.ihyj - (n.v000 - n.v0M0) * m.ihyjm) * m.ihfj;
    const T TN = (T(1) - m.thj) * n.uPM0 + m.thj * n.uP00, TS = (T(1) - m.thj) * n.u0M0 + m.thj * n.u000;
    const T QN = h * (n.v000 + n.vP00), QS = h * (n.vM00 + n.v000);
    cv += (TN * QN - TS * QS) * ihx;
    df += ((n.vP00 - n.v000) * ihx - (n.v000 - n.vM00) * ihx) * ihx;
    const T TT = (T(1) - m.thj) * n.w0MP + m.thj * n.w00P, TB = (T(1) - m.thj) * n.w0M0 + m.thj * n.w000;
    const T QT = h * (n.v000 + n.v00P), QB = h * (n.v00M + n.v000);
    cv += (TT * QT - TB * QB) * ihz;
    df += ((n.v00P - n.v000) * ihz - (n.v000 - n.v00M) * ihz) * ihz;
    Rv = -cv + nu * df;
  }
  {  // w on the z-face
    const T TE = h * (n.w000 + n.w00P), TW = h * (n.w00M + n.w000);
    T cv = (TE * TE - TW * TW) * ihz;
    T df = ((n.w00P - n.w000) * ihz - (n.w000 - n.w00M) * ihz) * ihz;
    const T TN = h * (n.uP0M + n.uP00), TS = h * (n.u00M + n.u000);
    const T QN = h * (n.w000 + n.wP00), QS = h * (n.wM00 + n.w000);
    cv += (TN * QN - TS * QS) * ihx;
    df += ((n.wP00 - n.w000) * ihx - (n.w000 - n.wM00) * ihx) * ihx;
    const T TT = h * (n.v0PM + n.v0P0), TB = h * (n.v00M + n.v000);
    const T QT = (T(1) - m.thjp) * n.w000 + m.thjp * n.w0P0, QB = (T(1) - m.thj) * n.w0M0 + m.thj * n.w000;
    cv += (TT * QT - TB * QB) * m.ihyj;
    df += ((n.w0P0 - n.w000) * m.ihfjp - (n.w000 - n.w0M0) * m.ihfj) * m.ihyj;
    Rw = -cv + nu * df;
  }
}

// Divergence of the Smagorinsky subgrid stress tau_ij = 2 nu_t S_ij on the three
// faces of a cell (uniform periodic grid): normal strains at the cell centres,
// shear strains at the edges, nu_t at centres (c) and averaged to edges (e*).
// nc: centres (i,j,k), (i-1), (j-1), (k-1); exy: edges (i,j), (i,j+1), (i+1,j);
// exz: (i,k), (i,k+1), (i+1,k); eyz: (j,k), (j,k+1), (j+1,k).
template <typename T>
__device__ __forceinline__ void sgs3(const Nb27<T>& n, const T* nc, const T* exy, const T* exz, const T* eyz,
                                     T ihx, T ihy, T ihz, T& Su, T& Sv, T& Sw) {
  const T h = T(0.5), two = T(2);
  // shear strains at the edges touching the cell's three faces
  const T sxy_ij = h * ((n.u000 - n.u0M0) * ihy + (n.v000 - n.vM00) * ihx);
  const T sxy_ijp = h * ((n.u0P0 - n.u000) * ihy + (n.v0P0 - n.vMP0) * ihx);
  const T sxy_ipj = h * ((n.uP00 - n.uPM0) * ihy + (n.vP00 - n.v000) * ihx);
  const T sxz_ik = h * ((n.u000 - n.u00M) * ihz + (n.w000 - n.wM00) * ihx);
  const T sxz_ikp = h * ((n.u00P - n.u000) * ihz + (n.w00P - n.wM0P) * ihx);
  const T sxz_ipk = h * ((n.uP00 - n.uP0M) * ihz + (n.wP00 - n.w000) * ihx);
  const T syz_jk = h * ((n.v000 - n.v00M) * ihz + (n.w000 - n.w0M0) * ihy);
  const T syz_jkp = h * ((n.v00P - n.v000) * ihz + (n.w00P - n.w0MP) * ihy);
  const T syz_jpk = h * ((n.v0P0 - n.v0PM) * ihz + (n.w0P0 - n.w000) * ihy);
  Su = (two * nc[0] * (n.uP00 - n.u000) * ihx - two * nc[1] * (n.u000 - n.uM00) * ihx) * ihx +
       (two * exy[1] * sxy_ijp - two * exy[0] * sxy_ij) * ihy + (two * exz[1] * sxz_ikp - two * exz[0] * sxz_ik) * ihz;
  Sv = (two * exy[2] * sxy_ipj - two * exy[0] * sxy_ij) * ihx +
       (two * nc[0] * (n.v0P0 - n.v000) * ihy - two * nc[2] * (n.v000 - n.v0M0) * ihy) * ihy +
       (two * eyz[1] * syz_jkp - two * eyz[0] * syz_jk) * ihz;
  Sw = (two * exz[2] * sxz_ipk - two * exz[0] * sxz_ik) * ihx + (two * eyz[2] * syz_jpk - two * eyz[0] * syz_jk) * ihy +
       (two * nc[0] * (n.w00P - n.w000) * ihz - two * nc[3] * (n.w000 - n.w00M) * ihz) * ihz;
}

// Eddy viscosity nu_t = (C_s Delta)^2 sqrt(2 S_ij S_ij) at cell (i, j, k) of a
// uniform periodic grid, the shear strains averaged from the four edges around
// the centre.
template <typename T>
__global__ void __launch_bounds__(kThreads) les_nut_kernel(const Geom<T> g, const T* __restrict__ U,
                                                           const T* __restrict__ V, const T* __restrict__ W,
                                                           T coef, T* __restrict__ nut) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if (i >= nx || j >= ny) return;
  const int xo[3] = {i > 0 ? i - 1 : nx - 1, i, i < nx - 1 ? i + 1 : 0};
  const int yo[3] = {j > 0 ? j - 1 : ny - 1, j, j < ny - 1 ? j + 1 : 0};
  const int zo[3] = {k > 0 ? k - 1 : nz - 1, k, k < nz - 1 ? k + 1 : 0};
  auto at = [&](int a, int b, int c) { return xo[a + 1] + nx * (yo[b + 1] + ny * zo[c + 1]); };
  const T ihx = g.ihx, ihy = g.ihy[0], ihz = g.ihz, h = T(0.5);
  const T sxx = (__ldg(U + at(1, 0, 0)) - __ldg(U + at(0, 0, 0))) * ihx;
  const T syy = (__ldg(V + at(0, 1, 0)) - __ldg(V + at(0, 0, 0))) * ihy;
  const T szz = (__ldg(W + at(0, 0, 1)) - __ldg(W + at(0, 0, 0))) * ihz;
  // edges (a, b) of a family at offsets a, b in {0, 1} from the cell's lower corner
  T cxy = T(0), cxz = T(0), cyz = T(0);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      cxy += h * ((__ldg(U + at(a, b, 0)) - __ldg(U + at(a, b - 1, 0))) * ihy +
                  (__ldg(V + at(a, b, 0)) - __ldg(V + at(a - 1, b, 0))) * ihx);
      cxz += h * ((__ldg(U + at(a, 0, b)) - __ldg(U + at(a, 0, b - 1))) * ihz +
                  (__ldg(W + at(a, 0, b)) - __ldg(W + at(a - 1, 0, b))) * ihx);
      cyz += h * ((__ldg(V + at(0, a, b)) - __ldg(V + at(0, a, b - 1))) * ihz +
                  (__ldg(W + at(0, a, b)) - __ldg(W + at(0, a - 1, b))) * ihy);
    }
  cxy *= T(0.25);
  cxz *= T(0.25);
  cyz *= T(0.25);
  const T ss = sxx * sxx + syy * syy + szz * szz + T(2) * (cxy * cxy + cxz * cxz + cyz * cyz);
  nut[at(0, 0, 0)] = coef * sqrt(T(2) * ss);
}

// nu_t averaged to the xy, xz and yz edges with the cell's index (lower corner).
template <typename T>
__global__ void __launch_bounds__(kThreads) les_edge_kernel(const Geom<T> g, const T* __restrict__ nut,
                                                            T* __restrict__ exy, T* __restrict__ exz,
                                                            T* __restrict__ eyz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if (i >= nx || j >= ny) return;
  const int im = i > 0 ? i - 1 : nx - 1, jm = j > 0 ? j - 1 : ny - 1, km = k > 0 ? k - 1 : nz - 1;
  auto c = [&](int a, int b, int d) { return __ldg(nut + a + nx * (b + ny * d)); };
  const T n0 = c(i, j, k), nxm = c(im, j, k), nym = c(i, jm, k), nzm = c(i, j, km);
  const size_t p = i + (size_t)nx * (j + (size_t)ny * k);
  exy[p] = T(0.25) * (n0 + nxm + nym + c(im, jm, k));
  exz[p] = T(0.25) * (n0 + nxm + nzm + c(im, j, km));
  eyz[p] = T(0.25) * (n0 + nym + nzm + c(i, jm, km));
}

// The general per-face path for the rows of a wall-bounded y whose stencil
// reaches a wall (j < 2 or j > ny - 2).
template <typename T>
__device__ __forceinline__ void predict_cell_general(const PredArgs<T>& A, int i, int j, int k) {
  const AccGhost<T> U{&A.g, A.uin, i, j, k};
  predict_face<T, 0>(A, U, i, j, k);
  predict_face<T, 1>(A, U, i, j, k);
  predict_face<T, 2>(A, U, i, j, k);
}

// The rows of a wall-bounded grid whose stencil reaches a wall (j = 0, 1, ny - 1,
// ny): one face per thread through the general path, launched beside the vector
// kernels, which then cover rows 2 .. ny - 2 only (a wall row inside a z-marching
// block would hold the whole block to the general path's pace).
template <typename T>
__global__ void __launch_bounds__(64) predictor_wall_rows_kernel(const PredArgs<T> A) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y / 3, c = blockIdx.y - 3 * r;   // row 0, 1, 2, 3 -> j = 0, 1, ny - 1, ny; component
  const int k = blockIdx.z;
  const int ny = A.g.ny;
  const int j = r < 2 ? r : ny - 3 + r;
  if (i >= A.X || j >= A.Y) return;
  const AccGhost<T> U{&A.g, A.uin, i, j, k};   // one face per thread
  if (c == 0) predict_face<T, 0>(A, U, i, j, k);
  else if (c == 1) predict_face<T, 1>(A, U, i, j, k);
  else predict_face<T, 2>(A, U, i, j, k);
}

// The predictor for the common 3-D case -- x and z periodic, central
// convection, no immersed body -- with the 27 distinct neighbour values of a
// cell loaded once and shared by its three faces.  YPER: y periodic (uniform
// metrics); otherwise y has walls and stretched metrics, and the rows whose
// stencil reaches a wall take the general path (j is warp-uniform: blocks are
// at least 32 wide in x).
template <typename T, bool YPER>
__global__ void __launch_bounds__(kThreads) predictor3_kernel(const PredArgs<T> A) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= A.X || j >= A.Y) return;
  const Geom<T>& g = A.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if (!YPER && (j < 2 || j > ny - 2)) {
    predict_cell_general(A, i, j, k);
    return;
  }
  const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
  const int km = k > 0 ? k - 1 : nz - 1, kp = k < nz - 1 ? k + 1 : 0;
  const int jm = YPER ? (j > 0 ? j - 1 : ny - 1) : j - 1;
  const int jp = YPER ? (j < ny - 1 ? j + 1 : 0) : j + 1;
  const int eyv = YPER ? ny : ny + 1;
  // row offsets of u, w (ny rows per plane) and v (eyv rows per plane)
  const int r00 = nx * (j + ny * k), rm0 = nx * (jm + ny * k), rp0 = nx * (jp + ny * k);
  const int r0m = nx * (j + ny * km), r0p = nx * (j + ny * kp), rmp = nx * (jm + ny * kp);
  const int v00 = nx * (j + eyv * k), vm0 = nx * (jm + eyv * k), vp0 = nx * (jp + eyv * k);
  const int v0m = nx * (j + eyv * km), v0p = nx * (j + eyv * kp), vpm = nx * (jp + eyv * km);
  const T* __restrict__ U = A.uin[0];
  const T* __restrict__ V = A.uin[1];
  const T* __restrict__ W = A.uin[2];
  Nb27<T> n;
  n.u000 = __ldg(U + r00 + i); n.uM00 = __ldg(U + r00 + im); n.uP00 = __ldg(U + r00 + ip);
  n.u0M0 = __ldg(U + rm0 + i); n.u0P0 = __ldg(U + rp0 + i); n.u00M = __ldg(U + r0m + i); n.u00P = __ldg(U + r0p + i);
  n.uPM0 = __ldg(U + rm0 + ip); n.uP0M = __ldg(U + r0m + ip);
  n.v000 = __ldg(V + v00 + i); n.vM00 = __ldg(V + v00 + im); n.vP00 = __ldg(V + v00 + ip);
  n.v0M0 = __ldg(V + vm0 + i); n.v0P0 = __ldg(V + vp0 + i); n.v00M = __ldg(V + v0m + i); n.v00P = __ldg(V + v0p + i);
  n.vMP0 = __ldg(V + vp0 + im); n.v0PM = __ldg(V + vpm + i);
  n.w000 = __ldg(W + r00 + i); n.wM00 = __ldg(W + r00 + im); n.wP00 = __ldg(W + r00 + ip);
  n.w0M0 = __ldg(W + rm0 + i); n.w0P0 = __ldg(W + rp0 + i); n.w00M = __ldg(W + r0m + i); n.w00P = __ldg(W + r0p + i);
  n.wM0P = __ldg(W + r0p + im); n.w0MP = __ldg(W + rmp + i);
  T Ru, Rv, Rw;
  rhs3(n, ymet<T, YPER>(A, j), g.ihx, g.ihz, g.nu, g.bforce ? g.bforce[j] : T(0), Ru, Rv, Rw);
  if (YPER && A.nut[0]) {   // Smagorinsky subgrid stress (uniform periodic grids)
    const int c00 = r00 + i;
    const T nc[4] = {__ldg(A.nut[0] + c00), __ldg(A.nut[0] + r00 + im), __ldg(A.nut[0] + rm0 + i),
                     __ldg(A.nut[0] + r0m + i)};
    const T exy[3] = {__ldg(A.nut[1] + c00), __ldg(A.nut[1] + rp0 + i), __ldg(A.nut[1] + r00 + ip)};
    const T exz[3] = {__ldg(A.nut[2] + c00), __ldg(A.nut[2] + r0p + i), __ldg(A.nut[2] + r00 + ip)};
    const T eyz[3] = {__ldg(A.nut[3] + c00), __ldg(A.nut[3] + r0p + i), __ldg(A.nut[3] + rp0 + i)};
    T Su, Sv, Sw;
    sgs3(n, nc, exy, exz, eyz, g.ihx, A.ihy0, g.ihz, Su, Sv, Sw);
    Ru += Su;
    Rv += Sv;
    Rw += Sw;
  }
  const T a = A.a, b = A.b, dt = A.dt;
  T ou = b * (n.u000 + dt * Ru), ov = b * (n.v000 + dt * Rv), ow = b * (n.w000 + dt * Rw);
  if (a != T(0)) {
    ou += a * A.un[0][r00 + i];
    ov += a * A.un[1][v00 + i];
    ow += a * A.un[2][r00 + i];
  }
  if (A.flags3[0]) {   // static 3-D body (forward Euler): u* = u_s = 0 and f on forced faces
    T fu = T(0), fv = T(0), fw = T(0);
    // the body is static: f is written on forced faces only and stays 0 elsewhere
    if (A.flags3[0][r00 + i]) { fu = -Ru - n.u000 / dt; ou = T(0); A.fout3[0][r00 + i] = fu; }
    if (A.flags3[1][v00 + i]) { fv = -Rv - n.v000 / dt; ov = T(0); A.fout3[1][v00 + i] = fv; }
    if (A.flags3[2][r00 + i]) { fw = -Rw - n.w000 / dt; ow = T(0); A.fout3[2][r00 + i] = fw; }
  }
  if (j < ny) {
    A.out[0][r00 + i] = ou;
    A.out[2][r00 + i] = ow;
  }
  A.out[1][v00 + i] = ov;
}

// VW consecutive floats (VW = 2 or 4) of a row whose start is 4 VW-byte aligned.
template <int VW>
__device__ __forceinline__ void ldw(const float* __restrict__ p, float* out) {
  if constexpr (VW == 4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
  } else {
    const float2 a = __ldg(reinterpret_cast<const float2*>(p));
    out[0] = a.x; out[1] = a.y;
  }
}
template <int VW>
__device__ __forceinline__ void stw(float* p, const float* in) {
  if constexpr (VW == 4) *reinterpret_cast<float4*>(p) = make_float4(in[0], in[1], in[2], in[3]);
  else *reinterpret_cast<float2*>(p) = make_float2(in[0], in[1]);
}

// Row segment of VW values at x = i0 .. i0+VW-1 with optional neighbours:
// s[0] = x[i0 - 1] (LO), s[1..VW] = x[i0 ..], s[VW + 1] = x[i0 + VW] (HI), periodic in x.
template <bool LO, bool HI, int VW>
__device__ __forceinline__ void ld_seg(const float* __restrict__ row, int i0, int nx, float* s) {
  ldw<VW>(row + i0, s + 1);
  if (LO) s[0] = __ldg(row + (i0 > 0 ? i0 - 1 : nx - 1));
  if (HI) s[VW + 1] = __ldg(row + (i0 + VW < nx ? i0 + VW : 0));
}

// VW cells per thread along x (FP32, nx % VW == 0, 4 VW-byte aligned fields):
// 17 VW-wide and 10 scalar loads feed the 3 x VW face updates.
template <bool YPER, int VW>
__global__ void __launch_bounds__(kThreads, 3) predictor3v_kernel(const PredArgs<float> A) {
  pdl_wait();
  const Geom<float>& g = A.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int i0 = VW * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = A.jlo + blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i0 >= nx || j >= A.Y) return;
  if (!YPER && (j < 2 || j > ny - 2)) {
    if (A.jlo > 0) return;   // the wall-row kernel has them
    for (int e = 0; e < VW; ++e) predict_cell_general(A, i0 + e, j, k);
    return;
  }
  const int km = k > 0 ? k - 1 : nz - 1, kp = k < nz - 1 ? k + 1 : 0;
  const int jm = YPER ? (j > 0 ? j - 1 : ny - 1) : j - 1;
  const int jp = YPER ? (j < ny - 1 ? j + 1 : 0) : j + 1;
  const int eyv = YPER ? ny : ny + 1;
  const int r00 = nx * (j + ny * k), rm0 = nx * (jm + ny * k), rp0 = nx * (jp + ny * k);
  const int r0m = nx * (j + ny * km), r0p = nx * (j + ny * kp), rmp = nx * (jm + ny * kp);
  const int v00 = nx * (j + eyv * k), vm0 = nx * (jm + eyv * k), vp0 = nx * (jp + eyv * k);
  const int v0m = nx * (j + eyv * km), v0p = nx * (j + eyv * kp), vpm = nx * (jp + eyv * km);
  const float* __restrict__ U = A.uin[0];
  const float* __restrict__ V = A.uin[1];
  const float* __restrict__ W = A.uin[2];
  constexpr int L = VW + 2;   // segments: index e + 1 is cell i0 + e
  float U00[L], UM0[L], UP0[L], U0M[L], U0P[L];
  float V00[L], VM0[L], VP0[L], V0M[L], V0P[L], VPM[L];
  float W00[L], WM0[L], WP0[L], W0M[L], W0P[L], WMP[L];
  ld_seg<true, true, VW>(U + r00, i0, nx, U00);
  ld_seg<false, true, VW>(U + rm0, i0, nx, UM0);
  ld_seg<false, false, VW>(U + rp0, i0, nx, UP0);
  ld_seg<false, true, VW>(U + r0m, i0, nx, U0M);
  ld_seg<false, false, VW>(U + r0p, i0, nx, U0P);
  ld_seg<true, true, VW>(V + v00, i0, nx, V00);
  ld_seg<false, false, VW>(V + vm0, i0, nx, VM0);
  ld_seg<true, false, VW>(V + vp0, i0, nx, VP0);
  ld_seg<false, false, VW>(V + v0m, i0, nx, V0M);
  ld_seg<false, false, VW>(V + v0p, i0, nx, V0P);
  ld_seg<false, false, VW>(V + vpm, i0, nx, VPM);
  ld_seg<true, true, VW>(W + r00, i0, nx, W00);
  ld_seg<false, false, VW>(W + rm0, i0, nx, WM0);
  ld_seg<false, false, VW>(W + rp0, i0, nx, WP0);
  ld_seg<false, false, VW>(W + r0m, i0, nx, W0M);
  ld_seg<true, false, VW>(W + r0p, i0, nx, W0P);
  ld_seg<false, false, VW>(W + rmp, i0, nx, WMP);
  const YMet<float> m = ymet<float, YPER>(A, j);
  const float bf = g.bforce ? g.bforce[j] : 0.f;
  const float a = A.a, b = A.b, dt = A.dt;
  float o3[3][VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    const int c = e + 1;
    Nb27<float> n;
    n.u000 = U00[c]; n.uM00 = U00[c - 1]; n.uP00 = U00[c + 1];
    n.u0M0 = UM0[c]; n.uPM0 = UM0[c + 1]; n.u0P0 = UP0[c];
    n.u00M = U0M[c]; n.uP0M = U0M[c + 1]; n.u00P = U0P[c];
    n.v000 = V00[c]; n.vM00 = V00[c - 1]; n.vP00 = V00[c + 1];
    n.v0M0 = VM0[c]; n.v0P0 = VP0[c]; n.vMP0 = VP0[c - 1];
    n.v00M = V0M[c]; n.v00P = V0P[c]; n.v0PM = VPM[c];
    n.w000 = W00[c]; n.wM00 = W00[c - 1]; n.wP00 = W00[c + 1];
    n.w0M0 = WM0[c]; n.w0P0 = WP0[c]; n.w00M = W0M[c];
    n.w00P = W0P[c]; n.wM0P = W0P[c - 1]; n.w0MP = WMP[c];
    float Ru, Rv, Rw;
    rhs3(n, m, g.ihx, g.ihz, g.nu, bf, Ru, Rv, Rw);
    o3[0][e] = b * (n.u000 + dt * Ru);
    o3[1][e] = b * (n.v000 + dt * Rv);
    o3[2][e] = b * (n.w000 + dt * Rw);
  }
  const int rows[3] = {r00, v00, r00};
  if (a != 0.f) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float pn[VW];
      ldw<VW>(A.un[c] + rows[c] + i0, pn);
#pragma unroll
      for (int e = 0; e < VW; ++e) o3[c][e] += a * pn[e];
    }
  }
  if (A.flags3[0]) {   // static 3-D body (forward Euler): u* = u_s = 0 and f on forced faces
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // u* = u + dt R, so R = (u* - u) / dt and f = -R - u / dt = -u* / dt; the body is
      // static, so f is written on forced faces only and stays 0 elsewhere
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        if (A.flags3[c][rows[c] + i0 + e]) {
          A.fout3[c][rows[c] + i0 + e] = -o3[c][e] / dt;
          o3[c][e] = 0.f;
        }
      }
    }
  }
  if (j < ny) {
    stw<VW>(A.out[0] + r00 + i0, o3[0]);
    stw<VW>(A.out[2] + r00 + i0, o3[2]);
  }
  stw<VW>(A.out[1] + v00 + i0, o3[1]);
}

// The 2-D counterpart for fully periodic uniform FP32 grids (no body): VW cells
// per thread along x, the arithmetic of Eq. (4) on the x- and y-faces with the
// uniform metrics (interpolation weights 1/2), six row segments per thread.
template <int VW>
__global__ void __launch_bounds__(kThreads) predictor2v_kernel(const PredArgs<float> A) {
  pdl_wait();
  const Geom<float>& g = A.g;
  const int nx = g.nx, ny = g.ny;
  const int i0 = VW * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i0 >= nx || j >= ny) return;
  const int jm = j > 0 ? j - 1 : ny - 1, jp = j < ny - 1 ? j + 1 : 0;
  const int r0 = nx * j, rm = nx * jm, rp = nx * jp;
  const float* __restrict__ U = A.uin[0];
  const float* __restrict__ V = A.uin[1];
  constexpr int L = VW + 2;   // index e + 1 is cell i0 + e
  float U0[L], UM[L], UP[L], V0[L], VM[L], VP[L];
  ld_seg<true, true, VW>(U + r0, i0, nx, U0);
  ld_seg<false, true, VW>(U + rm, i0, nx, UM);
  ld_seg<false, false, VW>(U + rp, i0, nx, UP);
  ld_seg<true, true, VW>(V + r0, i0, nx, V0);
  ld_seg<false, false, VW>(V + rm, i0, nx, VM);
  ld_seg<true, false, VW>(V + rp, i0, nx, VP);
  const float ihx = g.ihx, ihy = A.ihy0, nu = g.nu, h = 0.5f;
  const float bf = g.bforce ? g.bforce[j] : 0.f;
  const float a = A.a, b = A.b, dt = A.dt;
  float o2[2][VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    const int c = e + 1;
    const float u = U0[c], uW = U0[c - 1], uE = U0[c + 1], uS = UM[c], uN = UP[c], uSE = UM[c + 1];
    const float v = V0[c], vW = V0[c - 1], vE = V0[c + 1], vS = VM[c], vN = VP[c], vNW = VP[c - 1];
    // u on the x-face
    float TE = h * (u + uE), TW = h * (uW + u);
    float cv = (TE * TE - TW * TW) * ihx;
    float df = ((uE - u) * ihx - (u - uW) * ihx) * ihx;
    float TN = h * (vNW + vN), TS = h * (vW + v);
    cv += (TN * (h * (u + uN)) - TS * (h * (uS + u))) * ihy;
    df += ((uN - u) * ihy - (u - uS) * ihy) * ihy;
    const float Ru = -cv + nu * df + bf;
    // v on the y-face
    TE = h * (v + vN);
    TW = h * (vS + v);
    cv = (TE * TE - TW * TW) * ihy;
    df = ((vN - v) * ihy - (v - vS) * ihy) * ihy;
    TN = h * (uSE + uE);
    TS = h * (uS + u);
    cv += (TN * (h * (v + vE)) - TS * (h * (vW + v))) * ihx;
    df += ((vE - v) * ihx - (v - vW) * ihx) * ihx;
    const float Rv = -cv + nu * df;
    o2[0][e] = b * (u + dt * Ru);
    o2[1][e] = b * (v + dt * Rv);
  }
  if (a != 0.f) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float pn[VW];
      ldw<VW>(A.un[c] + r0 + i0, pn);
#pragma unroll
      for (int e = 0; e < VW; ++e) o2[c][e] += a * pn[e];
    }
  }
  stw<VW>(A.out[0] + r0 + i0, o2[0]);
  stw<VW>(A.out[1] + r0 + i0, o2[1]);
}

// The four-cell FP32 predictor marching in z: a thread computes the cells
// (i0 .. i0+3, j) of KZ consecutive planes, keeping the rows shared by
// neighbouring planes (the z neighbours of the stencil) in registers, so a plane
// takes 9 four-wide and 7 scalar loads instead of 17 and 10.
template <bool YPER>
__global__ void __launch_bounds__(kThreads, 2) predictor3z_kernel(const PredArgs<float> A, int KZ) {
  pdl_wait();
  const Geom<float>& g = A.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = A.jlo + blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * KZ;
  const int k1 = min(k0 + KZ, nz);
  if (i0 >= nx || j >= A.Y) return;
  if (!YPER && (j < 2 || j > ny - 2)) {
    if (A.jlo > 0) return;   // the wall-row kernel has them
    for (int k = k0; k < k1; ++k)
      for (int e = 0; e < 4; ++e) predict_cell_general(A, i0 + e, j, k);
    return;
  }
  const int jm = YPER ? (j > 0 ? j - 1 : ny - 1) : j - 1;
  const int jp = YPER ? (j < ny - 1 ? j + 1 : 0) : j + 1;
  const int eyv = YPER ? ny : ny + 1;
  auto ru = [&](int jj, int kk) { return nx * (jj + ny * kk); };
  auto rv = [&](int jj, int kk) { return nx * (jj + eyv * kk); };
  auto wrapk = [&](int kk) { return kk < 0 ? kk + nz : (kk >= nz ? kk - nz : kk); };
  const float* __restrict__ U = A.uin[0];
  const float* __restrict__ V = A.uin[1];
  const float* __restrict__ W = A.uin[2];
  constexpr int L = 6;
  // rows carried from plane to plane
  float Uc[L], Ukm[L], Vc[L], Vkm[L], Vpkm[L], Wc[L], Wmc[L], Wkm[L];
  {
    const int km = wrapk(k0 - 1);
    ld_seg<true, true, 4>(U + ru(j, k0), i0, nx, Uc);
    ld_seg<true, true, 4>(U + ru(j, km), i0, nx, Ukm);
    ld_seg<true, true, 4>(V + rv(j, k0), i0, nx, Vc);
    ld_seg<false, false, 4>(V + rv(j, km), i0, nx, Vkm);
    ld_seg<false, false, 4>(V + rv(jp, km), i0, nx, Vpkm);
    ld_seg<true, true, 4>(W + ru(j, k0), i0, nx, Wc);
    ld_seg<false, false, 4>(W + ru(jm, k0), i0, nx, Wmc);
    ld_seg<false, false, 4>(W + ru(j, km), i0, nx, Wkm);
  }
  const YMet<float> m = ymet<float, YPER>(A, j);
  const float bf = g.bforce ? g.bforce[j] : 0.f;
  const float a = A.a, b = A.b, dt = A.dt;
  for (int k = k0; k < k1; ++k) {
    const int kp = wrapk(k + 1);
    float UM0[L], UP0[L], U0P[L], VM0[L], VP0[L], V0P[L], WP0[L], W0P[L], WMP[L];
    ld_seg<false, true, 4>(U + ru(jm, k), i0, nx, UM0);
    ld_seg<false, false, 4>(U + ru(jp, k), i0, nx, UP0);
    ld_seg<true, true, 4>(U + ru(j, kp), i0, nx, U0P);
    ld_seg<false, false, 4>(V + rv(jm, k), i0, nx, VM0);
    ld_seg<true, false, 4>(V + rv(jp, k), i0, nx, VP0);
    ld_seg<true, true, 4>(V + rv(j, kp), i0, nx, V0P);
    ld_seg<false, false, 4>(W + ru(jp, k), i0, nx, WP0);
    ld_seg<true, true, 4>(W + ru(j, kp), i0, nx, W0P);
    ld_seg<false, false, 4>(W + ru(jm, kp), i0, nx, WMP);
    const int rows[3] = {ru(j, k), rv(j, k), ru(j, k)};
    // the RK stage's u^n rows, issued with the stencil rows (one memory round trip per plane)
    float pn[3][4];
    if (a != 0.f) {
#pragma unroll
      for (int c = 0; c < 3; ++c) ldw<4>(A.un[c] + rows[c] + i0, pn[c]);
    }
    float o3[3][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int c = e + 1;
      Nb27<float> n;
      n.u000 = Uc[c]; n.uM00 = Uc[c - 1]; n.uP00 = Uc[c + 1];
      n.u0M0 = UM0[c]; n.uPM0 = UM0[c + 1]; n.u0P0 = UP0[c];
      n.u00M = Ukm[c]; n.uP0M = Ukm[c + 1]; n.u00P = U0P[c];
      n.v000 = Vc[c]; n.vM00 = Vc[c - 1]; n.vP00 = Vc[c + 1];
      n.v0M0 = VM0[c]; n.v0P0 = VP0[c]; n.vMP0 = VP0[c - 1];
      n.v00M = Vkm[c]; n.v00P = V0P[c]; n.v0PM = Vpkm[c];
      n.w000 = Wc[c]; n.wM00 = Wc[c - 1]; n.wP00 = Wc[c + 1];
      n.w0M0 = Wmc[c]; n.w0P0 = WP0[c]; n.w00M = Wkm[c];
      n.w00P = W0P[c]; n.wM0P = W0P[c - 1]; n.w0MP = WMP[c];
      float Ru, Rv, Rw;
      rhs3(n, m, g.ihx, g.ihz, g.nu, bf, Ru, Rv, Rw);
      o3[0][e] = b * (n.u000 + dt * Ru);
      o3[1][e] = b * (n.v000 + dt * Rv);
      o3[2][e] = b * (n.w000 + dt * Rw);
    }
    if (a != 0.f) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) o3[c][e] += a * pn[c][e];
    }
    if (A.flags3[0]) {   // static 3-D body (forward Euler): u* = u_s = 0 and f on forced faces
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const uchar4 fl = *reinterpret_cast<const uchar4*>(A.flags3[c] + rows[c] + i0);
        const bool on[4] = {fl.x != 0, fl.y != 0, fl.z != 0, fl.w != 0};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (on[e]) {   // f on forced faces only (static body: 0 elsewhere from the start)
            A.fout3[c][rows[c] + i0 + e] = -o3[c][e] / dt;
            o3[c][e] = 0.f;
          }
        }
      }
    }
    if (j < ny) {
      stw<4>(A.out[0] + rows[0] + i0, o3[0]);
      stw<4>(A.out[2] + rows[2] + i0, o3[2]);
    }
    stw<4>(A.out[1] + rows[1] + i0, o3[1]);
    // next plane: the centre rows move to k - 1, the k + 1 rows to the centre
#pragma unroll
    for (int q = 0; q < L; ++q) {
      Ukm[q] = Uc[q];
      Uc[q] = U0P[q];
      Vkm[q] = Vc[q];
      Vpkm[q] = VP0[q];
      Vc[q] = V0P[q];
      Wkm[q] = Wc[q];
      Wc[q] = W0P[q];
      Wmc[q] = WMP[q];
    }
  }
}

// Staged z-marching predictor: fully periodic uniform FP32 grids with nx = NX
// (128 or 256).  A block works on the whole x extent of BY = 1024 / NX rows
// j0 .. j0+BY-1 and a run of consecutive planes.  On grids that stay in L2 the
// launch holds two blocks per SM and gives each an equal share of the (row
// block, plane) units, a run split where it crosses into the next row block.
// On larger grids (chunk > 0) every row block is cut into the same runs of
// `chunk` planes and the blocks of neighbouring row blocks, adjacent in launch
// order, march the same planes together, so that the y halo rows a block
// stages were brought into L2 by its neighbours (equal shares start their runs
// at unrelated planes and read those rows again from DRAM: 30.7 against 24 B
// per cell at 256^3).  One thread streams each plane's U,
// V and W rows j0-1 .. j0+BY (periodic y halo) from global to shared memory with
// bulk asynchronous copies into a ring of plane slots, up to four planes
// ahead of the compute; a staged plane serves the iterations of its own plane
// and of its two z neighbours.  Each thread computes four cells of one row from
// shared memory (x neighbours wrap inside the row); the RK stage's u^n and the
// outputs go through plain vector loads and stores.
//
// Arithmetic: the central divergence-form convection of Eq. (4) on a uniform
// grid, written with the face sums s = u_a + u_b (the halves of Eq. 4's
// interpolations folded into the factor 1/4) and one product per cell edge.
// The product at an edge serves the two faces that share it: the lower xy edge
// of cell e is the x flux of v at e and e - 1 and the lower y flux of u; the
// products of the x edges are shared by the four cells of a thread, and those
// of the z-upper edges and faces are carried to the next plane as its lower
// ones.  Diffusion is the uniform second difference.
template <int NX>
struct StageGeo {
  static constexpr int TX = NX / 4;       // threads per row
  static constexpr int BY = 1024 / NX;    // rows per block (256 threads)
  static constexpr int RR = BY + 2;       // rows per staged slab (y halo)
  static constexpr int FIELD = RR * NX;   // floats per field in a slot
  static constexpr int SLOT = 3 * FIELD;  // floats per slot
  static constexpr int RING = NX == 128 ? 7 : 5;   // plane slots: RING - 3 planes in flight ahead
};

template <int NX>
constexpr size_t stage_smem() {
  return (size_t)StageGeo<NX>::RING * StageGeo<NX>::SLOT * sizeof(float);
}

// s[0] = row[i0 - 1] (LO), s[1..4] = row[i0 .. i0+3], s[5] = row[i0 + 4] (HI), periodic in x
template <bool LO, bool HI, int NX>
__device__ __forceinline__ void lds_seg(const float* row, int i0, float* s) {
  const float4 a = *reinterpret_cast<const float4*>(row + i0);
  s[1] = a.x; s[2] = a.y; s[3] = a.z; s[4] = a.w;
  if (LO) s[0] = row[(i0 - 1) & (NX - 1)];
  if (HI) s[5] = row[(i0 + 4) & (NX - 1)];
}

template <int NX>
__global__ void __launch_bounds__(kThreads, 2) predictor3t_kernel(const PredArgs<float> A, unsigned* status, int chunk) {
  using SG = StageGeo<NX>;
  extern __shared__ __align__(16) float stg[];
  constexpr int kStageRing = SG::RING;
  __shared__ uint64_t bars[kStageRing];
  pdl_wait();
  const Geom<float>& g = A.g;
  const int ny = g.ny, nz = g.nz;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool leader = tx == 0 && ty == 0;
  if (leader) {
    for (int s = 0; s < kStageRing; ++s) mbar_init(&bars[s], 1);
    mbar_init_fence();
  }
  // the block's share of the (row block, plane) units, in row-block-major order: a
  // contiguous run of planes, split where it crosses into the next row block
  const int nyb = (ny + SG::BY - 1) / SG::BY;
  const long long total = (long long)nyb * nz;
  int u0, u1;
  if (chunk > 0) {   // aligned runs: row block fastest in launch order
    const int rb = blockIdx.x % nyb, ch = blockIdx.x / nyb;
    u0 = rb * nz + ch * chunk;
    u1 = rb * nz + min((ch + 1) * chunk, nz);
  } else {
    u0 = (int)(total * blockIdx.x / gridDim.x);
    u1 = (int)(total * (blockIdx.x + 1) / gridDim.x);
  }
  const int i0 = 4 * tx;
  const int rm = ty * NX, r0 = (ty + 1) * NX, rp = (ty + 2) * NX;
  const float a = A.a, b = A.b, dt = A.dt, nu = g.nu;
  const float ihx = g.ihx, ihy = A.ihy0, ihz = g.ihz;
  const float qx = 0.25f * ihx, qy = 0.25f * ihy, qz = 0.25f * ihz;
  const float dx2 = ihx * ihx, dy2 = ihy * ihy, dz2 = ihz * ihz, d0 = -2.f * (dx2 + dy2 + dz2);
  bool ok = true;
  int base = 0;   // planes this block has staged so far: ring slot and phase of the next one
  for (int u = u0; u < u1;) {
  const int yb = u / nz;
  const int k0 = u - yb * nz;
  const int kz = min(nz - k0, u1 - u);   // planes computed in this run
  u += kz;
  const int j0 = yb * SG::BY;
  const int nplanes = kz + 2;        // planes staged: k0 - 1 .. k0 + kz
  __syncthreads();   // barriers initialised; every slot of the previous run consumed
  // slab row r holds y row (j0 - 1 + r) mod ny: at most two contiguous runs (ny >= RR)
  const int g0 = j0 == 0 ? ny - 1 : j0 - 1;
  const int run1 = min(SG::RR, ny - g0);
  auto issue = [&](int rel) {   // stage plane k0 - 1 + rel (leader only)
    int p = k0 - 1 + rel;
    p = p < 0 ? p + nz : (p >= nz ? p - nz : p);
    const int s = (base + rel) % kStageRing;
    float* slot = stg + (size_t)s * SG::SLOT;
    mbar_expect_tx(&bars[s], SG::SLOT * sizeof(float));
    for (int f = 0; f < 3; ++f) {
      const float* src = A.uin[f] + (size_t)p * ny * NX;
      float* dst = slot + f * SG::FIELD;
      bulk_g2s(dst, src + (size_t)g0 * NX, run1 * NX * sizeof(float), &bars[s]);
      if (run1 < SG::RR) bulk_g2s(dst + run1 * NX, src, (SG::RR - run1) * NX * sizeof(float), &bars[s]);
    }
  };
  if (leader)
    for (int rel = 0; rel < kStageRing - 1 && rel < nplanes; ++rel) issue(rel);
  auto wait = [&](int rel) {
    ok = mbar_wait(&bars[(base + rel) % kStageRing], ((base + rel) / kStageRing) & 1) && ok;
  };
  auto slotp = [&](int rel) { return stg + (size_t)((base + rel) % kStageRing) * SG::SLOT; };
  const int j = j0 + ty;
  const bool act = j < ny;
  const float bf = g.bforce ? g.bforce[act ? j : 0] : 0.f;
  // products of the lower z edges / faces of the current plane, carried from plane to plane
  float Exz[5], Eyz[4], Szz[4];
  wait(0);
  wait(1);
  {
    const float* Pm = slotp(0);   // plane k0 - 1
    const float* P0 = slotp(1);   // plane k0
    float Ukm[6], Uc[6], Wc[6], Vkm[6], Vc[6], Wmc[6], Wkm[6];
    lds_seg<false, true, NX>(Pm + r0, i0, Ukm);
    lds_seg<false, true, NX>(P0 + r0, i0, Uc);
    lds_seg<true, true, NX>(P0 + 2 * SG::FIELD + r0, i0, Wc);
    lds_seg<false, false, NX>(Pm + SG::FIELD + r0, i0, Vkm);
    lds_seg<false, false, NX>(P0 + SG::FIELD + r0, i0, Vc);
    lds_seg<false, false, NX>(P0 + 2 * SG::FIELD + rm, i0, Wmc);
    lds_seg<false, false, NX>(Pm + 2 * SG::FIELD + r0, i0, Wkm);
#pragma unroll
    for (int e = 0; e < 5; ++e) Exz[e] = (Ukm[e + 1] + Uc[e + 1]) * (Wc[e] + Wc[e + 1]);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      Eyz[e] = (Vkm[e + 1] + Vc[e + 1]) * (Wmc[e + 1] + Wc[e + 1]);
      const float t = Wkm[e + 1] + Wc[e + 1];
      Szz[e] = t * t;
    }
  }
  for (int kk = 0; kk < kz; ++kk) {
    const int k = k0 + kk;
    __syncthreads();   // the slot of plane kk - 1 is free
    if (leader && kk + kStageRing - 1 < nplanes) issue(kk + kStageRing - 1);
    const size_t row = (size_t)NX * (j + (size_t)ny * k);
    float pn[3][4];
    if (a != 0.f && act) {
#pragma unroll
      for (int c = 0; c < 3; ++c) ldw<4>(A.un[c] + row + i0, pn[c]);
    }
    wait(kk + 2);
    const float* Pm = slotp(kk);       // plane k - 1
    const float* P0 = slotp(kk + 1);   // plane k
    const float* Pp = slotp(kk + 2);   // plane k + 1
    const float* U0 = P0;
    const float* V0 = P0 + SG::FIELD;
    const float* W0 = P0 + 2 * SG::FIELD;
    float Uc[6], UM0[6], UP0[6], Ukm[6], U0P[6];
    float Vc[6], VM0[6], VP0[6], Vkm[6], V0P[6], Vpkm[6];
    float Wc[6], Wmc[6], WP0[6], Wkm[6], W0P[6], WMP[6];
    lds_seg<true, true, NX>(U0 + r0, i0, Uc);
    lds_seg<false, true, NX>(U0 + rm, i0, UM0);
    lds_seg<false, false, NX>(U0 + rp, i0, UP0);
    lds_seg<false, false, NX>(Pm + r0, i0, Ukm);
    lds_seg<false, true, NX>(Pp + r0, i0, U0P);
    lds_seg<true, true, NX>(V0 + r0, i0, Vc);
    lds_seg<false, false, NX>(V0 + rm, i0, VM0);
    lds_seg<true, false, NX>(V0 + rp, i0, VP0);
    lds_seg<false, false, NX>(Pm + SG::FIELD + r0, i0, Vkm);
    lds_seg<false, false, NX>(Pp + SG::FIELD + r0, i0, V0P);
    lds_seg<false, false, NX>(Pm + SG::FIELD + rp, i0, Vpkm);
    lds_seg<true, true, NX>(W0 + r0, i0, Wc);
    lds_seg<false, false, NX>(W0 + rm, i0, Wmc);
    lds_seg<false, false, NX>(W0 + rp, i0, WP0);
    lds_seg<false, false, NX>(Pm + 2 * SG::FIELD + r0, i0, Wkm);
    lds_seg<true, true, NX>(Pp + 2 * SG::FIELD + r0, i0, W0P);
    lds_seg<false, false, NX>(Pp + 2 * SG::FIELD + rm, i0, WMP);
    // edge and face products of this plane (x edges: five for four cells) and of the z-upper ones
    float sq[5], Exy[5], Exz_up[5], Eyz_up[4], Szz_up[4];
#pragma unroll
    for (int e = 0; e < 5; ++e) {
      const float su = Uc[e] + Uc[e + 1];
      sq[e] = su * su;
      Exy[e] = (UM0[e + 1] + Uc[e + 1]) * (Vc[e] + Vc[e + 1]);
      Exz_up[e] = (Uc[e + 1] + U0P[e + 1]) * (W0P[e] + W0P[e + 1]);
    }
    float o3[3][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int c = e + 1;
      Eyz_up[e] = (Vc[c] + V0P[c]) * (WMP[c] + W0P[c]);
      const float tz = Wc[c] + W0P[c];
      Szz_up[e] = tz * tz;
      const float Nxy = (VP0[e] + VP0[c]) * (Uc[c] + UP0[c]);
      const float Nyz = (Vpkm[c] + VP0[c]) * (Wc[c] + WP0[c]);
      const float vn = Vc[c] + VP0[c], vs = VM0[c] + Vc[c];
      // u on the x face
      float cv = qx * (sq[c] - sq[e]);
      cv = fmaf(qy, Nxy - Exy[e], cv);
      cv = fmaf(qz, Exz_up[e] - Exz[e], cv);
      float df = fmaf(d0, Uc[c], dx2 * (Uc[e] + Uc[c + 1]));
      df = fmaf(dy2, UM0[c] + UP0[c], df);
      df = fmaf(dz2, Ukm[c] + U0P[c], df);
      const float Ru = fmaf(nu, df, bf - cv);
      // v on the y face
      cv = qy * (vn * vn - vs * vs);
      cv = fmaf(qx, Exy[c] - Exy[e], cv);
      cv = fmaf(qz, Eyz_up[e] - Eyz[e], cv);
      df = fmaf(d0, Vc[c], dx2 * (Vc[e] + Vc[c + 1]));
      df = fmaf(dy2, VM0[c] + VP0[c], df);
      df = fmaf(dz2, Vkm[c] + V0P[c], df);
      const float Rv = fmaf(nu, df, -cv);
      // w on the z face
      cv = qz * (Szz_up[e] - Szz[e]);
      cv = fmaf(qx, Exz[c] - Exz[e], cv);
      cv = fmaf(qy, Nyz - Eyz[e], cv);
      df = fmaf(d0, Wc[c], dx2 * (Wc[e] + Wc[c + 1]));
      df = fmaf(dy2, Wmc[c] + WP0[c], df);
      df = fmaf(dz2, Wkm[c] + W0P[c], df);
      const float Rw = fmaf(nu, df, -cv);
      o3[0][e] = b * fmaf(dt, Ru, Uc[c]);
      o3[1][e] = b * fmaf(dt, Rv, Vc[c]);
      o3[2][e] = b * fmaf(dt, Rw, Wc[c]);
    }
#pragma unroll
    for (int e = 0; e < 5; ++e) Exz[e] = Exz_up[e];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      Eyz[e] = Eyz_up[e];
      Szz[e] = Szz_up[e];
    }
    if (act) {
      if (a != 0.f) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int e = 0; e < 4; ++e) o3[c][e] = fmaf(a, pn[c][e], o3[c][e]);
      }
      if (A.flags3[0]) {   // static 3-D body (forward Euler): u* = u_s = 0 and f on forced faces
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const uchar4 fl = *reinterpret_cast<const uchar4*>(A.flags3[c] + row + i0);
          const bool on[4] = {fl.x != 0, fl.y != 0, fl.z != 0, fl.w != 0};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (on[e]) {   // f on forced faces only (static body: 0 elsewhere from the start)
              A.fout3[c][row + i0 + e] = -o3[c][e] / dt;
              o3[c][e] = 0.f;
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) stw<4>(A.out[c] + row + i0, o3[c]);
    }
  }
  base += nplanes;
  }
  if (!ok) atomicOr(status, 1u);   // a staged plane never arrived: results of this block are invalid
}

template <typename T>
__global__ void outflow_scale_kernel(const T* __restrict__ u0, int ex, int ny, int nz, const double* __restrict__ hy,
                                     double hz, double q_in, double* scale) {
  __shared__ double sh[kThreads];
  pdl_wait();
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
__global__ void __launch_bounds__(kThreads) divergence_kernel(const DivArgs<T> A, T* __restrict__ out) {
  const Geom<T>& g = A.g;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  out[i + g.nx * (j + g.ny * k)] = div_at(A, i, j, k);
}

template <typename T>
struct CorrArgs {
  Geom<T> g;
  const T* us[3];
  const T* phi;
  T* un[3];
  int X, Y;
};

template <typename T, int C>
__device__ __forceinline__ void correct_face(const CorrArgs<T>& A, int i, int j, int k, const T phi0) {
  const Geom<T>& g = A.g;
  const int ex = g.ext(C, 0), ey = g.ext(C, 1), ez = g.ext(C, 2);
  if (i >= ex || j >= ey || k >= ez) return;
  const int t = i + ex * (j + ey * k);
  int idx[3] = {i, j, k};
  const int nC = (C == 0) ? g.nx : (C == 1 ? g.ny : g.nz);
  T v = A.us[C][t];
  if (g.per[C] || (idx[C] > 0 && idx[C] < nC)) {
    // G phi at the face: (phi[cell f] - phi[cell f-1]) / hf
    int lo[3] = {i, j, k};
    lo[C] = idx[C] > 0 ? idx[C] - 1 : nC - 1;
    const int c1 = lo[0] + g.nx * (lo[1] + g.ny * lo[2]);
    const T ihf = (C == 0) ? g.ihx : (C == 1 ? g.ihfy[j] : g.ihz);
    v -= (phi0 - __ldg(A.phi + c1)) * ihf;
  }
  A.un[C][t] = v;
}

// Eq. (10): u^{n+1} = u* - G phi on every interior face; one thread per cell position.
template <typename T>
__global__ void __launch_bounds__(kThreads) correct_kernel(const CorrArgs<T> A) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= A.X || j >= A.Y) return;
  const Geom<T>& g = A.g;
  const bool in_cells = i < g.nx && j < g.ny;
  const T phi0 = in_cells ? __ldg(A.phi + i + g.nx * (j + g.ny * k)) : T(0);
  correct_face<T, 0>(A, i, j, k, phi0);
  correct_face<T, 1>(A, i, j, k, phi0);
  if (g.dim == 3) correct_face<T, 2>(A, i, j, k, phi0);
}

// Eq. (10) for grids with periodic x and nx % 4 == 0: four cells per thread,
// row-vector loads and stores (y faces on walls keep their imposed value).
template <typename T>
__global__ void __launch_bounds__(kThreads) correct4_kernel(const CorrArgs<T> A) {
  pdl_wait();
  const Geom<T>& g = A.g;
  const int nx = g.nx, ny = g.ny;
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i0 >= nx || j >= A.Y) return;
  const bool cell = j < ny;
  const size_t rowc = (size_t)nx * (j + (size_t)ny * k);
  Vec4<T> p0 = {{T(0), T(0), T(0), T(0)}};
  if (cell) {
    p0 = ld4(A.phi + rowc + i0);
    const T pm = __ldg(A.phi + rowc + (i0 > 0 ? i0 - 1 : nx - 1));
    Vec4<T> a = ld4(A.us[0] + rowc + i0);
    a.v[0] -= (p0.v[0] - pm) * g.ihx;
    a.v[1] -= (p0.v[1] - p0.v[0]) * g.ihx;
    a.v[2] -= (p0.v[2] - p0.v[1]) * g.ihx;
    a.v[3] -= (p0.v[3] - p0.v[2]) * g.ihx;
    st4(A.un[0] + rowc + i0, a);
  }
  {
    const int ey = g.ext(1, 1);
    const size_t t = (size_t)nx * (j + (size_t)ey * k) + i0;
    Vec4<T> a = ld4(A.us[1] + t);
    if (g.per[1] || (j > 0 && j < ny)) {
      const int jm = j > 0 ? j - 1 : ny - 1;
      const Vec4<T> pm = ld4(A.phi + (size_t)nx * (jm + (size_t)ny * k) + i0);
      const T ih = g.ihfy[j];
#pragma unroll
      for (int e = 0; e < 4; ++e) a.v[e] -= (p0.v[e] - pm.v[e]) * ih;
    }
    st4(A.un[1] + t, a);
  }
  if (g.dim == 3 && cell) {
    const int km = k > 0 ? k - 1 : g.nz - 1;
    const Vec4<T> pm = ld4(A.phi + (size_t)nx * (j + (size_t)ny * km) + i0);
    Vec4<T> a = ld4(A.us[2] + rowc + i0);
#pragma unroll
    for (int e = 0; e < 4; ++e) a.v[e] -= (p0.v[e] - pm.v[e]) * g.ihz;
    st4(A.un[2] + rowc + i0, a);
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
  for (int c = 0; c < 3; ++c) {
    const bool on = c < G->dim;
    A.uin[c] = on ? uin[c] : nullptr;
    A.un[c] = (on && un) ? un[c] : nullptr;
    A.out[c] = on ? out[c] : nullptr;
  }
  A.dt = (T)dt;
  A.a = (T)a;
  A.b = (T)b;
  A.conv = G->conv;
  A.X = G->nx + (G->per[0] ? 0 : 1);
  A.Y = G->ny + (G->per[1] ? 0 : 1);
  A.jlo = 0;
  for (int c = 0; c < 2; ++c) {
    const bool ibc = G->has_body;
    A.flags[c] = ibc ? G->ib.flags[c] : nullptr;
    A.num[c] = ibc ? (T*)G->ib.num[c] : nullptr;
    A.den[c] = ibc ? (T*)G->ib.den[c] : nullptr;
    A.fout[c] = ibc ? (T*)G->ib.f[c] : nullptr;
  }
  A.body = body_state;
  A.omega = G->ib.omega;
  A.cx = G->ib.centre[0];
  A.cy = G->ib.centre[1];
  A.xf = G->xf64[0];
  A.yf = G->xf64[1];
  A.oscale = G->scal;
  A.ihy0 = (T)(1.0 / G->h[1][0]);
  for (int c = 0; c < 3; ++c) {
    A.flags3[c] = G->has_ib3 ? G->ib3.flags[c] : nullptr;
    A.fout3[c] = G->has_ib3 ? (T*)G->ib3.f[c] : nullptr;
  }
  const bool les = G->les_cs > 0.0;
  for (int q = 0; q < 4; ++q) A.nut[q] = les ? (const T*)G->les_nu[q] : nullptr;
  if (les) {
    const Geom<T> gg = G->geom<T>();
    double delta = std::cbrt(G->hx * G->h[1][0] * G->hz);
    const T coef = (T)(G->les_cs * delta * G->les_cs * delta);
    const dim3 lb = stencil_block(G), lg = stencil_grid(G, G->nx, G->ny);
    launch_pdl(G, "les_nut", les_nut_kernel<T>, lg, lb, 0, gg, (const T*)uin[0], (const T*)uin[1], (const T*)uin[2],
               coef, (T*)G->les_nu[0]);
    FS_LAUNCH(G, "les_nut", les_edge_kernel<T><<<lg, lb, 0, G->stream>>>(gg, (const T*)G->les_nu[0], (T*)G->les_nu[1],
                                                                       (T*)G->les_nu[2], (T*)G->les_nu[3]));
  }
  const dim3 blk = stencil_block(G);
  const dim3 grd = stencil_grid(G, A.X, A.Y);
  if (G->dim == 3 && G->per[0] && G->per[2] && G->conv == FS_CENTRAL2 && !G->has_body && G->ny >= 4) {
    if (les) {   // the one-cell kernel carries the subgrid term
      launch_pdl(G, "predictor", predictor3_kernel<T, true>, grd, blk, 0, A);
      return;
    }
    if constexpr (std::is_same<T, float>::value) {
      const int vw = G->tune_pred_vw > 0 ? G->tune_pred_vw : 4;
      bool vec = vw > 1 && G->nx % vw == 0;   // 1: the one-cell kernel
      for (int c = 0; c < 3; ++c) {
        vec = vec && (uintptr_t)uin[c] % (4 * vw) == 0 && (uintptr_t)out[c] % (4 * vw) == 0;
        if (un) vec = vec && (uintptr_t)un[c] % (4 * vw) == 0;
        if (G->has_ib3) vec = vec && (uintptr_t)G->ib3.f[c] % (4 * vw) == 0;
      }
      const int KZ = G->tune_zmarch > 0 ? G->tune_zmarch : 8;
      const int nx = G->nx;
      if (vec && vw == 4 && G->tune_staged && G->per[1] && (nx == 128 || nx == 256) && G->ny >= 1024 / nx + 2) {
        static bool attr = false;
        if (!attr) {
          cudaFuncSetAttribute(predictor3t_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)stage_smem<128>());
          cudaFuncSetAttribute(predictor3t_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)stage_smem<256>());
          attr = true;
        }
        static int nsm = 0;
        if (!nsm) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
        const int by = 1024 / nx;
        const int nyb = (G->ny + by - 1) / by;
        const long long units = (long long)nyb * G->nz;
        // L2-resident grids (three velocity fields within half of the 126 MB L2): two resident
        // blocks per SM, each with an equal share of the (row block, plane) units; larger grids:
        // runs of `chunk` planes aligned across row blocks, about two blocks per SM in one wave
        int chunk = G->tune_pred_chunk;
        if (chunk == 0 && (size_t)3 * sizeof(float) * G->nx * G->ny * G->nz > (size_t)64 << 20) {
          const int runs = std::max(1, 2 * std::max(nsm, 1) / nyb);
          chunk = (G->nz + runs - 1) / runs;
        }
        if (chunk < 0) chunk = 0;
        const dim3 sg = chunk > 0 ? dim3((unsigned)(nyb * ((G->nz + chunk - 1) / chunk)))
                                  : dim3((unsigned)std::min<long long>(units, 2LL * std::max(nsm, 1)));
        if (nx == 128)
          launch_pdl(G, "predictor", predictor3t_kernel<128>, sg, dim3(32, 8), stage_smem<128>(), A, G->dstatus, chunk);
        else
          launch_pdl(G, "predictor", predictor3t_kernel<256>, sg, dim3(64, 4), stage_smem<256>(), A, G->dstatus, chunk);
        return;
      }
      // walls: the four rows that reach a wall run in their own kernel, the vector kernels take rows 2 .. ny - 2
      int rows = A.Y;
      if (vec && !G->per[1] && G->ny >= 5) {
        A.jlo = 2;
        rows = G->ny - 3;
        launch_pdl(G, "predictor_walls", predictor_wall_rows_kernel<T>, dim3((A.X + 63) / 64, 12, G->nz), dim3(64), 0,
                   A);
      }
      if (vec && vw == 4 && KZ > 1) {
        const dim3 vb(32, 8);
        const dim3 vg((G->nx / 4 + 31) / 32, (rows + 7) / 8, (G->nz + KZ - 1) / KZ);
        if (G->per[1]) launch_pdl(G, "predictor", predictor3z_kernel<true>, vg, vb, 0, A, KZ);
        else launch_pdl(G, "predictor", predictor3z_kernel<false>, vg, vb, 0, A, KZ);
        return;
      }
      if (vec) {
        const dim3 vb(32, 8);
        const dim3 vg((G->nx / vw + 31) / 32, (rows + 7) / 8, G->nz);
        if (vw == 4) {
          if (G->per[1]) launch_pdl(G, "predictor", predictor3v_kernel<true, 4>, vg, vb, 0, A);
          else launch_pdl(G, "predictor", predictor3v_kernel<false, 4>, vg, vb, 0, A);
        } else {
          if (G->per[1]) launch_pdl(G, "predictor", predictor3v_kernel<true, 2>, vg, vb, 0, A);
          else launch_pdl(G, "predictor", predictor3v_kernel<false, 2>, vg, vb, 0, A);
        }
        return;
      }
    }
    if (G->per[1])
      launch_pdl(G, "predictor", predictor3_kernel<T, true>, grd, blk, 0, A);
    else
      launch_pdl(G, "predictor", predictor3_kernel<T, false>, grd, blk, 0, A);
    return;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (G->dim == 2 && G->per[0] && G->per[1] && G->conv == FS_CENTRAL2 && !G->has_body && G->nx % 4 == 0 &&
        G->tune_pred_vw != 1) {
      bool vec = true;
      for (int c = 0; c < 2; ++c) {
        vec = vec && (uintptr_t)uin[c] % 16 == 0 && (uintptr_t)out[c] % 16 == 0;
        if (un) vec = vec && (uintptr_t)un[c] % 16 == 0;
      }
      if (vec) {
        const dim3 vb(32, 8), vg((G->nx / 4 + 31) / 32, (G->ny + 7) / 8);
        launch_pdl(G, "predictor", predictor2v_kernel<4>, vg, vb, 0, A);
        return;
      }
    }
  }
  launch_pdl(G, "predictor", predictor_kernel<T>, grd, blk, 0, A);
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
  launch_pdl(G, "outflow_scale", outflow_scale_kernel<T>, dim3(1), dim3(kThreads), 0, (const T*)uin[0], G->nx + 1,
             G->ny, G->nz, (const double*)G->hy64, G->dim == 3 ? G->hz : 1.0, q_in, (double*)G->scal);
}

template <typename T>
DivArgs<T> make_div_args(fs_grid* G, T* const* u, const double* body_state) {
  DivArgs<T> A;
  A.g = G->geom<T>();
  for (int c = 0; c < 3; ++c) A.u[c] = c < G->dim ? u[c] : nullptr;
  A.flags[0] = G->has_body ? G->ib.flags[0] : nullptr;
  A.flags[1] = G->has_body ? G->ib.flags[1] : nullptr;
  A.body = body_state;
  A.omega = G->ib.omega;
  A.cx = G->ib.centre[0];
  A.cy = G->ib.centre[1];
  A.xf = G->xf64[0];
  A.yf = G->xf64[1];
  A.vec4 = (G->per[0] && G->nx % 4 == 0 && !G->has_body) ? 1 : 0;
  for (int c = 0; c < G->dim; ++c)
    if ((uintptr_t)u[c] % (4 * sizeof(T))) A.vec4 = 0;
  return A;
}

template <typename T>
void launch_divergence(fs_grid* G, T* const* u, T* out, const double* body_state) {
  const DivArgs<T> A = make_div_args<T>(G, u, body_state);
  const dim3 blk = stencil_block(G);
  const dim3 grd = stencil_grid(G, G->nx, G->ny);
  FS_LAUNCH(G, "divergence", divergence_kernel<T><<<grd, blk, 0, G->stream>>>(A, out));
}

template <typename T>
void launch_correct(fs_grid* G, T* const* ustar, const T* phi, T* const* unew) {
  CorrArgs<T> A;
  A.g = G->geom<T>();
  for (int c = 0; c < 3; ++c) {
    A.us[c] = c < G->dim ? ustar[c] : nullptr;
    A.un[c] = c < G->dim ? unew[c] : nullptr;
  }
  A.phi = phi;
  A.X = G->nx + (G->per[0] ? 0 : 1);
  A.Y = G->ny + (G->per[1] ? 0 : 1);
  bool vec = G->per[0] && G->nx % 4 == 0 && (uintptr_t)phi % (4 * sizeof(T)) == 0;
  for (int c = 0; c < G->dim; ++c)
    vec = vec && (uintptr_t)ustar[c] % (4 * sizeof(T)) == 0 && (uintptr_t)unew[c] % (4 * sizeof(T)) == 0;
  if (vec) {
    const dim3 blk(32, 8);
    const dim3 grd((G->nx / 4 + 31) / 32, (A.Y + 7) / 8, G->nz);
    launch_pdl(G, "correct", correct4_kernel<T>, grd, blk, 0, A);
    return;
  }
  const dim3 blk = stencil_block(G);
  const dim3 grd = stencil_grid(G, A.X, A.Y);
  launch_pdl(G, "correct", correct_kernel<T>, grd, blk, 0, A);
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
  template DivArgs<T> make_div_args<T>(fs_grid*, T* const*, const double*);                                     \
  template void launch_correct<T>(fs_grid*, T* const*, const T*, T* const*);                                     \
  template void launch_to_pressure<T>(fs_grid*, const T*, double*, double);                                      \
  template void launch_diagnostics<T>(fs_grid*, T* const*, double*);
FS_INST(float)
FS_INST(double)
#undef FS_INST

}  // namespace fs
