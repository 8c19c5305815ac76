// Discrete adjoint of one time step (fs_step_adjoint), §2.4.1 of the paper:
// the paper differentiates its solver by reverse-mode AD; this file is the
// hand-written transpose of every kernel of the forward step, so
//   lam^n = (d step / d state^n)^T lam^{n+1}   (plus parameter gradients).
//
//   predictor   R'(u)^T mu: the exact reverse of the per-face forward flux
//               computation, scattered to the faces it read (ghost rules
//               transposed), plus the direct-forcing and RK terms
//   projection  P^T = I - D^T V S V^-1 G^T (L = D G is symmetric in the
//               cell-volume inner product), the same direct Poisson solver S
//   outflow     transpose of the flux-balanced zero-gradient face
//   IB          force spreading transposed (marker -> grid), the marker
//               position derivative through phi'(r); the epsilon mask is
//               frozen (its derivative is zero almost everywhere)
//   body        reverse of the four RK4 stages, d/dk accumulated (FP64)
//
// Adjoint fields have the precision of the grid's fields; gradient
// accumulators and body adjoints are FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "fs_internal.cuh"

namespace fs {

namespace {

constexpr int kT = 256;

// Transpose of ldv: add v to the adjoint of the stored value that ldv would
// read at (i, j, k) for component c; imposed boundary values absorb nothing.
template <typename T>
__device__ __forceinline__ void adj_add(const Geom<T>& g, T* __restrict__ lam, int c, int i, int j, int k, T v) {
  int idx[3] = {i, j, k};
  int e[3] = {g.ext(c, 0), g.ext(c, 1), g.ext(c, 2)};
  T sign = T(1);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int q = idx[d];
    if (q < 0 || q >= e[d]) {
      const int side = q < 0 ? 0 : 1;
      if (g.per[d]) {
        q = side ? q - e[d] : q + e[d];
      } else {
        q = side ? e[d] - 1 : 0;
        if (d != c && bc_dirichlet(g.bc[d][side])) sign = -sign;
      }
      idx[d] = q;
    }
  }
  const int own = idx[c];
  if (!g.per[c] && (own == 0 || own == e[c] - 1) && g.bc[c][own == 0 ? 0 : 1] != FS_BC_OUTFLOW) return;
  atomicAdd(lam + idx[0] + e[0] * (idx[1] + e[1] * idx[2]), sign * v);
}

// Reverse of momentum_rhs for the C-face (i, j, k): adds (dR/du)^T * gm to lam.
template <typename T, int C>
__device__ __forceinline__ void rhs_adjoint_face(const Geom<T>& g, const T* const* u, T* const* lam, int conv,
                                                 int i, int j, int k, T gm) {
  const int idx[3] = {i, j, k};
  constexpr int cx = C == 0, cy = C == 1, cz = C == 2;
  {
    const T uW = ldv(g, u[C], C, i - cx, j - cy, k - cz);
    const T u0 = ldv(g, u[C], C, i, j, k);
    const T uE = ldv(g, u[C], C, i + cx, j + cy, k + cz);
    const T TE = T(0.5) * (u0 + uE), TW = T(0.5) * (uW + u0);
    T ihf, ihE, ihW;
    if (C == 1) {
      ihf = g.ihfy[j];
      ihE = g.ihy[j < g.ny ? j : g.ny - 1];
      ihW = g.ihy[j > 0 ? j - 1 : (g.per[1] ? g.ny - 1 : 0)];
    } else {
      ihf = ihE = ihW = (C == 0) ? g.ihx : g.ihz;
    }
    // R = -(TE QE - TW QW) ihf + nu ((uE - u0) ihE - (u0 - uW) ihW) ihf
    const T gE = -gm * ihf, gW = gm * ihf;   // adjoints of TE*QE and TW*QW
    T aW = T(0), a0 = T(0), aE = T(0);
    if (conv == FS_UPWIND1) {
      const T QE = TE > T(0) ? u0 : uE, QW = TW > T(0) ? uW : u0;
      a0 += T(0.5) * gE * QE;
      aE += T(0.5) * gE * QE;
      if (TE > T(0)) a0 += gE * TE; else aE += gE * TE;
      aW += T(0.5) * gW * QW;
      a0 += T(0.5) * gW * QW;
      if (TW > T(0)) aW += gW * TW; else a0 += gW * TW;
    } else {
      a0 += gE * TE + gW * TW;     // d(T^2) = 2 T dT, dT = (du0 + duE) / 2
      aE += gE * TE;
      aW += gW * TW;
    }
    const T nd = gm * g.nu * ihf;
    aE += nd * ihE;
    a0 -= nd * (ihE + ihW);
    aW += nd * ihW;
    adj_add(g, lam[C], C, i - cx, j - cy, k - cz, aW);
    adj_add(g, lam[C], C, i, j, k, a0);
    adj_add(g, lam[C], C, i + cx, j + cy, k + cz, aE);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d == C || d >= g.dim) continue;
    const int dx = d == 0, dy = d == 1, dz = d == 2;
    const T thc = (C == 1) ? g.thy[j] : T(0.5);
    const T A1 = ldv(g, u[d], d, i + dx - cx, j + dy - cy, k + dz - cz);
    const T A2 = ldv(g, u[d], d, i + dx, j + dy, k + dz);
    const T B1 = ldv(g, u[d], d, i - cx, j - cy, k - cz);
    const T B2 = ldv(g, u[d], d, i, j, k);
    const T TN = (T(1) - thc) * A1 + thc * A2;
    const T TS = (T(1) - thc) * B1 + thc * B2;
    const T uS = ldv(g, u[C], C, i - dx, j - dy, k - dz);
    const T u0 = ldv(g, u[C], C, i, j, k);
    const T uN = ldv(g, u[C], C, i + dx, j + dy, k + dz);
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
    // R = -(TN QN - TS QS) ihd + nu ((uN - u0) ihfN - (u0 - uS) ihfS) ihd
    const T gN = -gm * ihd, gS = gm * ihd;
    const T gTN = gN * QN, gQN = gN * TN, gTS = gS * QS, gQS = gS * TS;
    adj_add(g, lam[d], d, i + dx - cx, j + dy - cy, k + dz - cz, (T(1) - thc) * gTN);
    adj_add(g, lam[d], d, i + dx, j + dy, k + dz, thc * gTN);
    adj_add(g, lam[d], d, i - cx, j - cy, k - cz, (T(1) - thc) * gTS);
    adj_add(g, lam[d], d, i, j, k, thc * gTS);
    T aS = T(0), a0 = T(0), aN = T(0);
    if (conv == FS_UPWIND1) {
      if (TN > T(0)) a0 += gQN; else aN += gQN;
      if (TS > T(0)) aS += gQS; else a0 += gQS;
    } else {
      a0 += (T(1) - thN) * gQN + thS * gQS;
      aN += thN * gQN;
      aS += (T(1) - thS) * gQS;
    }
    const T nd = gm * g.nu * ihd;
    aN += nd * ihfN;
    a0 -= nd * (ihfN + ihfS);
    aS += nd * ihfS;
    adj_add(g, lam[C], C, i - dx, j - dy, k - dz, aS);
    adj_add(g, lam[C], C, i, j, k, a0);
    adj_add(g, lam[C], C, i + dx, j + dy, k + dz, aN);
  }
}

template <typename T>
struct RhsAdjArgs {
  Geom<T> g;
  const T* u[3];     // state the forward R was evaluated at
  const T* mu[3];    // adjoint of R on each face (0 on boundary faces)
  T* lam[3];         // receives R'(u)^T mu
  int conv;
  int X, Y;
};

template <typename T>
__global__ void __launch_bounds__(kT) rhs_adjoint_kernel(const RhsAdjArgs<T> A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= A.X || j >= A.Y) return;
  const Geom<T>& g = A.g;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (c >= g.dim) break;
    const int ex = g.ext(c, 0), ey = g.ext(c, 1), ez = g.ext(c, 2);
    if (i >= ex || j >= ey || k >= ez) continue;
    const T gm = A.mu[c][i + ex * (j + ey * k)];
    if (gm == T(0)) continue;
    if (c == 0) rhs_adjoint_face<T, 0>(g, A.u, A.lam, A.conv, i, j, k, gm);
    else if (c == 1) rhs_adjoint_face<T, 1>(g, A.u, A.lam, A.conv, i, j, k, gm);
    else rhs_adjoint_face<T, 2>(g, A.u, A.lam, A.conv, i, j, k, gm);
  }
}

// Gather form of rhs_adjoint for fully periodic 3-D grids with central
// convection (uniform metrics): every thread forms lam(p) += (dR/du(p))^T mu
// for the three faces at its cell p from the flux adjoints of all fluxes that
// read u(p), so no atomics are needed.  With R_C(f) = -(F(f) - F(f - e)) i_e per
// flux F on the interface between faces f and f + e, the flux adjoint is
// aF(f) = i_e (mu_C(f + e) - mu_C(f)); the own-direction flux F = T^2,
// T = (u_C(f) + u_C(f + e_C)) / 2, gives aF T to both faces, and the cross flux
// E_Cd(f) = TN QN, TN = (u_d(f + e_d - e_C) + u_d(f + e_d)) / 2,
// QN = (u_C(f) + u_C(f + e_d)) / 2, gives aE TN / 2 to the two u_C and aE QN / 2
// to the two u_d it reads.  Diffusion is symmetric on a uniform periodic grid.
// out = src + R'(u)^T (scale src): the gather below evaluated on mu = scale src.
template <typename T>
struct GatherAdjArgs {
  RhsAdjArgs<T> r;   // u, mu = src, g
  T scale;
  T* out[3];
  const T* add[3];   // added to out (the RK stage accumulator of the last stage), or null
};

// The neighbour values one cell's gather reads (u, v, w: linearisation point; m*: mu).
template <typename T>
struct AdjNb {
  T u0, uPx, uMx, uMy, uPxMy, uMz, uPxMz;
  T v0, vPy, vMx, vMxPy, vMy, vMz, vPyMz;
  T w0, wPz, wMx, wMxPz, wMy, wMyPz, wMz;
  T mu0, muPx, muMx, muPy, muMy, muPz, muMz, muPxMy, muPxMz;
  T mv0, mvPy, mvPx, mvMx, mvMxPy, mvMy, mvPz, mvMz, mvPyMz;
  T mw0, mwPz, mwPx, mwMx, mwMxPz, mwPy, mwMy, mwMyPz, mwMz;
};

// (dR/du)^T mu at the three faces of one cell (see rhs_adjoint_gather_kernel).
template <typename T>
__device__ __forceinline__ void gather_adj_cell(const AdjNb<T>& n, T ihx, T ihy, T ihz, T nu, T& lu, T& lv, T& lw) {
  const T h = T(0.5);
  {  // lambda_u
    T l = ihx * (n.muPx - n.mu0) * h * (n.u0 + n.uPx) + ihx * (n.mu0 - n.muMx) * h * (n.uMx + n.u0);
    l += h * (ihy * (n.muPy - n.mu0) * h * (n.vMxPy + n.vPy) + ihy * (n.mu0 - n.muMy) * h * (n.vMx + n.v0));
    l += h * (ihz * (n.muPz - n.mu0) * h * (n.wMxPz + n.wPz) + ihz * (n.mu0 - n.muMz) * h * (n.wMx + n.w0));
    l += h * (ihx * (n.mvPy - n.mvMxPy) * h * (n.vMxPy + n.vPy) + ihx * (n.mv0 - n.mvMx) * h * (n.vMx + n.v0));
    l += h * (ihx * (n.mwPz - n.mwMxPz) * h * (n.wMxPz + n.wPz) + ihx * (n.mw0 - n.mwMx) * h * (n.wMx + n.w0));
    l += nu * ((n.muPx - T(2) * n.mu0 + n.muMx) * ihx * ihx + (n.muPy - T(2) * n.mu0 + n.muMy) * ihy * ihy +
               (n.muPz - T(2) * n.mu0 + n.muMz) * ihz * ihz);
    lu = l;
  }
  {  // lambda_v
    T l = ihy * (n.mvPy - n.mv0) * h * (n.v0 + n.vPy) + ihy * (n.mv0 - n.mvMy) * h * (n.vMy + n.v0);
    l += h * (ihx * (n.mvPx - n.mv0) * h * (n.uPxMy + n.uPx) + ihx * (n.mv0 - n.mvMx) * h * (n.uMy + n.u0));
    l += h * (ihz * (n.mvPz - n.mv0) * h * (n.wMyPz + n.wPz) + ihz * (n.mv0 - n.mvMz) * h * (n.wMy + n.w0));
    l += h * (ihy * (n.muPx - n.muPxMy) * h * (n.uPxMy + n.uPx) + ihy * (n.mu0 - n.muMy) * h * (n.uMy + n.u0));
    l += h * (ihy * (n.mwPz - n.mwMyPz) * h * (n.wMyPz + n.wPz) + ihy * (n.mw0 - n.mwMy) * h * (n.wMy + n.w0));
    l += nu * ((n.mvPx - T(2) * n.mv0 + n.mvMx) * ihx * ihx + (n.mvPy - T(2) * n.mv0 + n.mvMy) * ihy * ihy +
               (n.mvPz - T(2) * n.mv0 + n.mvMz) * ihz * ihz);
    lv = l;
  }
  {  // lambda_w
    T l = ihz * (n.mwPz - n.mw0) * h * (n.w0 + n.wPz) + ihz * (n.mw0 - n.mwMz) * h * (n.wMz + n.w0);
    l += h * (ihx * (n.mwPx - n.mw0) * h * (n.uPxMz + n.uPx) + ihx * (n.mw0 - n.mwMx) * h * (n.uMz + n.u0));
    l += h * (ihy * (n.mwPy - n.mw0) * h * (n.vPyMz + n.vPy) + ihy * (n.mw0 - n.mwMy) * h * (n.vMz + n.v0));
    l += h * (ihz * (n.muPx - n.muPxMz) * h * (n.uPxMz + n.uPx) + ihz * (n.mu0 - n.muMz) * h * (n.uMz + n.u0));
    l += h * (ihz * (n.mvPy - n.mvPyMz) * h * (n.vPyMz + n.vPy) + ihz * (n.mv0 - n.mvMz) * h * (n.vMz + n.v0));
    l += nu * ((n.mwPx - T(2) * n.mw0 + n.mwMx) * ihx * ihx + (n.mwPy - T(2) * n.mw0 + n.mwMy) * ihy * ihy +
               (n.mwPz - T(2) * n.mw0 + n.mwMz) * ihz * ihz);
    lw = l;
  }
}

template <typename T>
__global__ void __launch_bounds__(kT) rhs_adjoint_gather_kernel(const GatherAdjArgs<T> GA) {
  const RhsAdjArgs<T>& A = GA.r;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  const Geom<T>& g = A.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if (i >= nx || j >= ny) return;
  const int xo[3] = {i > 0 ? i - 1 : nx - 1, i, i < nx - 1 ? i + 1 : 0};
  const int yo[3] = {j > 0 ? j - 1 : ny - 1, j, j < ny - 1 ? j + 1 : 0};
  const int zo[3] = {k > 0 ? k - 1 : nz - 1, k, k < nz - 1 ? k + 1 : 0};
  auto at = [&](int di, int dj, int dk) { return xo[di + 1] + nx * (yo[dj + 1] + ny * zo[dk + 1]); };
  auto ld = [&](const T* f, int a, int b, int c) { return __ldg(f + at(a, b, c)); };
  const T *U = A.u[0], *V = A.u[1], *W = A.u[2], *MU = A.mu[0], *MV = A.mu[1], *MW = A.mu[2];
  AdjNb<T> n;
  n.u0 = ld(U, 0, 0, 0); n.uPx = ld(U, 1, 0, 0); n.uMx = ld(U, -1, 0, 0); n.uMy = ld(U, 0, -1, 0);
  n.uPxMy = ld(U, 1, -1, 0); n.uMz = ld(U, 0, 0, -1); n.uPxMz = ld(U, 1, 0, -1);
  n.v0 = ld(V, 0, 0, 0); n.vPy = ld(V, 0, 1, 0); n.vMx = ld(V, -1, 0, 0); n.vMxPy = ld(V, -1, 1, 0);
  n.vMy = ld(V, 0, -1, 0); n.vMz = ld(V, 0, 0, -1); n.vPyMz = ld(V, 0, 1, -1);
  n.w0 = ld(W, 0, 0, 0); n.wPz = ld(W, 0, 0, 1); n.wMx = ld(W, -1, 0, 0); n.wMxPz = ld(W, -1, 0, 1);
  n.wMy = ld(W, 0, -1, 0); n.wMyPz = ld(W, 0, -1, 1); n.wMz = ld(W, 0, 0, -1);
  n.mu0 = ld(MU, 0, 0, 0); n.muPx = ld(MU, 1, 0, 0); n.muMx = ld(MU, -1, 0, 0); n.muPy = ld(MU, 0, 1, 0);
  n.muMy = ld(MU, 0, -1, 0); n.muPz = ld(MU, 0, 0, 1); n.muMz = ld(MU, 0, 0, -1); n.muPxMy = ld(MU, 1, -1, 0);
  n.muPxMz = ld(MU, 1, 0, -1);
  n.mv0 = ld(MV, 0, 0, 0); n.mvPy = ld(MV, 0, 1, 0); n.mvPx = ld(MV, 1, 0, 0); n.mvMx = ld(MV, -1, 0, 0);
  n.mvMxPy = ld(MV, -1, 1, 0); n.mvMy = ld(MV, 0, -1, 0); n.mvPz = ld(MV, 0, 0, 1); n.mvMz = ld(MV, 0, 0, -1);
  n.mvPyMz = ld(MV, 0, 1, -1);
  n.mw0 = ld(MW, 0, 0, 0); n.mwPz = ld(MW, 0, 0, 1); n.mwPx = ld(MW, 1, 0, 0); n.mwMx = ld(MW, -1, 0, 0);
  n.mwMxPz = ld(MW, -1, 0, 1); n.mwPy = ld(MW, 0, 1, 0); n.mwMy = ld(MW, 0, -1, 0); n.mwMyPz = ld(MW, 0, -1, 1);
  n.mwMz = ld(MW, 0, 0, -1);
  T lu, lv, lw;
  gather_adj_cell(n, g.ihx, g.ihy[0], g.ihz, g.nu, lu, lv, lw);
  const int p = at(0, 0, 0);
  T o0 = n.mu0 + GA.scale * lu, o1 = n.mv0 + GA.scale * lv, o2 = n.mw0 + GA.scale * lw;
  if (GA.add[0]) {
    o0 += GA.add[0][p];
    o1 += GA.add[1][p];
    o2 += GA.add[2][p];
  }
  GA.out[0][p] = o0;
  GA.out[1][p] = o1;
  GA.out[2][p] = o2;
}

// Four cells per thread along x (FP32, n_x % 4 == 0, 16-byte aligned fields): the
// rows of the 30 neighbour segments are read as float4 vectors plus the x
// neighbours they need, then the per-cell gather above.
__device__ __forceinline__ void ld4s(const float* __restrict__ row, int i0, int nx, float* s, bool lo, bool hi) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(row + i0));
  s[1] = a.x; s[2] = a.y; s[3] = a.z; s[4] = a.w;
  s[0] = lo ? __ldg(row + (i0 > 0 ? i0 - 1 : nx - 1)) : 0.f;
  s[5] = hi ? __ldg(row + (i0 + 4 < nx ? i0 + 4 : 0)) : 0.f;
}

__global__ void __launch_bounds__(kT, 2) rhs_adjoint_gather4_kernel(const GatherAdjArgs<float> GA) {
  const RhsAdjArgs<float>& A = GA.r;
  const Geom<float>& g = A.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i0 >= nx || j >= ny) return;
  const int jm = j > 0 ? j - 1 : ny - 1, jp = j < ny - 1 ? j + 1 : 0;
  const int km = k > 0 ? k - 1 : nz - 1, kp = k < nz - 1 ? k + 1 : 0;
  auto row = [&](const float* f, int jj, int kk) { return f + (size_t)nx * (jj + (size_t)ny * kk); };
  const float *U = A.u[0], *V = A.u[1], *W = A.u[2], *MU = A.mu[0], *MV = A.mu[1], *MW = A.mu[2];
  float u00[6], um0[6], u0m[6];
  float v00[6], vp0[6], vm0[6], v0m[6], vpm[6];
  float w00[6], w0p[6], wm0[6], wmp[6], w0m[6];
  float mu00[6], mup0[6], mum0[6], mu0p[6], mu0m[6];
  float mv00[6], mvp0[6], mvm0[6], mv0p[6], mv0m[6], mvpm[6];
  float mw00[6], mw0p[6], mwp0[6], mwmp[6], mwm0[6], mw0m[6];
  ld4s(row(U, j, k), i0, nx, u00, true, true);
  ld4s(row(U, jm, k), i0, nx, um0, false, true);
  ld4s(row(U, j, km), i0, nx, u0m, false, true);
  ld4s(row(V, j, k), i0, nx, v00, true, false);
  ld4s(row(V, jp, k), i0, nx, vp0, true, false);
  ld4s(row(V, jm, k), i0, nx, vm0, false, false);
  ld4s(row(V, j, km), i0, nx, v0m, false, false);
  ld4s(row(V, jp, km), i0, nx, vpm, false, false);
  ld4s(row(W, j, k), i0, nx, w00, true, false);
  ld4s(row(W, j, kp), i0, nx, w0p, true, false);
  ld4s(row(W, jm, k), i0, nx, wm0, false, false);
  ld4s(row(W, jm, kp), i0, nx, wmp, false, false);
  ld4s(row(W, j, km), i0, nx, w0m, false, false);
  ld4s(row(MU, j, k), i0, nx, mu00, true, true);
  ld4s(row(MU, jp, k), i0, nx, mup0, false, false);
  ld4s(row(MU, jm, k), i0, nx, mum0, false, true);
  ld4s(row(MU, j, kp), i0, nx, mu0p, false, false);
  ld4s(row(MU, j, km), i0, nx, mu0m, false, true);
  ld4s(row(MV, j, k), i0, nx, mv00, true, true);
  ld4s(row(MV, jp, k), i0, nx, mvp0, true, false);
  ld4s(row(MV, jm, k), i0, nx, mvm0, false, false);
  ld4s(row(MV, j, kp), i0, nx, mv0p, false, false);
  ld4s(row(MV, j, km), i0, nx, mv0m, false, false);
  ld4s(row(MV, jp, km), i0, nx, mvpm, false, false);
  ld4s(row(MW, j, k), i0, nx, mw00, true, true);
  ld4s(row(MW, j, kp), i0, nx, mw0p, true, false);
  ld4s(row(MW, jp, k), i0, nx, mwp0, false, false);
  ld4s(row(MW, jm, kp), i0, nx, mwmp, false, false);
  ld4s(row(MW, jm, k), i0, nx, mwm0, false, false);
  ld4s(row(MW, j, km), i0, nx, mw0m, false, false);
  float o[3][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int c = e + 1;
    AdjNb<float> n;
    n.u0 = u00[c]; n.uPx = u00[c + 1]; n.uMx = u00[c - 1]; n.uMy = um0[c]; n.uPxMy = um0[c + 1];
    n.uMz = u0m[c]; n.uPxMz = u0m[c + 1];
    n.v0 = v00[c]; n.vPy = vp0[c]; n.vMx = v00[c - 1]; n.vMxPy = vp0[c - 1]; n.vMy = vm0[c]; n.vMz = v0m[c];
    n.vPyMz = vpm[c];
    n.w0 = w00[c]; n.wPz = w0p[c]; n.wMx = w00[c - 1]; n.wMxPz = w0p[c - 1]; n.wMy = wm0[c]; n.wMyPz = wmp[c];
    n.wMz = w0m[c];
    n.mu0 = mu00[c]; n.muPx = mu00[c + 1]; n.muMx = mu00[c - 1]; n.muPy = mup0[c]; n.muMy = mum0[c];
    n.muPz = mu0p[c]; n.muMz = mu0m[c]; n.muPxMy = mum0[c + 1]; n.muPxMz = mu0m[c + 1];
    n.mv0 = mv00[c]; n.mvPy = mvp0[c]; n.mvPx = mv00[c + 1]; n.mvMx = mv00[c - 1]; n.mvMxPy = mvp0[c - 1];
    n.mvMy = mvm0[c]; n.mvPz = mv0p[c]; n.mvMz = mv0m[c]; n.mvPyMz = mvpm[c];
    n.mw0 = mw00[c]; n.mwPz = mw0p[c]; n.mwPx = mw00[c + 1]; n.mwMx = mw00[c - 1]; n.mwMxPz = mw0p[c - 1];
    n.mwPy = mwp0[c]; n.mwMy = mwm0[c]; n.mwMyPz = mwmp[c]; n.mwMz = mw0m[c];
    float lu, lv, lw;
    gather_adj_cell(n, g.ihx, g.ihy[0], g.ihz, g.nu, lu, lv, lw);
    o[0][e] = n.mu0 + GA.scale * lu;
    o[1][e] = n.mv0 + GA.scale * lv;
    o[2][e] = n.mw0 + GA.scale * lw;
  }
  const size_t p = (size_t)nx * (j + (size_t)ny * k) + i0;
  if (GA.add[0]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(GA.add[c] + p));
      o[c][0] += a.x;
      o[c][1] += a.y;
      o[c][2] += a.z;
      o[c][3] += a.w;
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) *reinterpret_cast<float4*>(GA.out[c] + p) = make_float4(o[c][0], o[c][1], o[c][2], o[c][3]);
}

// x = -(G^T lam) / V at every cell: the right-hand side of the adjoint Poisson solve.
template <typename T>
__global__ void __launch_bounds__(kT) adj_rhs_kernel(const Geom<T> g, const T* __restrict__ l0,
                                                     const T* __restrict__ l1, const T* __restrict__ l2,
                                                     const double* __restrict__ hy, T* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const T* L[3] = {l0, l1, l2};
  const int n[3] = {g.nx, g.ny, g.nz};
  const int p[3] = {i, j, k};
  T gt = T(0);
  for (int c = 0; c < g.dim; ++c) {
    const int ex = g.ext(c, 0), ey = g.ext(c, 1);
    // face f = cell (left face) and f + 1 (right face) along c
    const bool lo_in = g.per[c] || p[c] > 0;
    const bool hi_in = g.per[c] || p[c] + 1 < n[c];
    int q[3] = {i, j, k};
    const T ihf_lo = c == 0 ? g.ihx : (c == 1 ? g.ihfy[j] : g.ihz);
    if (lo_in) gt += L[c][q[0] + ex * (q[1] + ey * q[2])] * ihf_lo;
    q[c] = p[c] + 1;
    if (g.per[c] && q[c] == n[c]) q[c] = 0;
    const T ihf_hi = c == 0 ? g.ihx : (c == 1 ? g.ihfy[j + 1] : g.ihz);
    if (hi_in) gt -= L[c][q[0] + ex * (q[1] + ey * q[2])] * ihf_hi;
  }
  const double V = (double)g.hx * hy[j] * (g.dim == 3 ? (double)g.hz : 1.0);
  out[i + g.nx * (j + g.ny * k)] = T(-(double)gt / V);
}

// lam~ on face f of component c: D^T (V y) = A(f-1) y[f-1] - A(f) y[f], A = V / h_c.
template <typename T>
__device__ __forceinline__ T adj_div_T(const Geom<T>& g, const T* __restrict__ y, const double* __restrict__ hy,
                                       int c, int i, int j, int k) {
  const int n[3] = {g.nx, g.ny, g.nz};
  const int p[3] = {i, j, k};
  const double hz = g.dim == 3 ? (double)g.hz : 1.0;
  double r = 0.0;
  // cell f - 1 (left of the face)
  int q[3] = {i, j, k};
  bool have = true;
  if (p[c] == 0) {
    if (g.per[c]) q[c] = n[c] - 1; else have = false;
  } else {
    q[c] = p[c] - 1;
  }
  auto area = [&](int jj) {
    if (c == 0) return hy[jj] * hz;
    if (c == 1) return (double)g.hx * hz;
    return (double)g.hx * hy[jj];
  };
  if (have) r += area(q[1]) * (double)y[q[0] + g.nx * (q[1] + g.ny * q[2])];
  if (p[c] < n[c]) r -= area(j) * (double)y[i + g.nx * (j + g.ny * k)];
  return T(r);
}

// Per-face adjoint of projection + predictor (forward Euler, optional body).
template <typename T>
struct FaceAdjArgs {
  Geom<T> g;
  const T* lam1[3];      // lambda of u^{n+1}
  const T* y;            // adjoint pressure (solved)
  const double* hy;
  T dt;
  // forward Euler with body
  const uint8_t* flags[2];
  const T* lamf[2];      // adjoint of the forcing term f (forced faces)
  double* wdsum;         // [2] accumulators: adjoint of the body velocity (FP64)
  double* bfsum;         // [ny] accumulators: adjoint of the body-force profile, or null
  T* mu[3];              // out: adjoint of R (0 on boundary faces)
  T* lamn[3];            // out: direct part of lambda of u^n
  T* lamout;             // out: lambda of u* on the outflow faces [nz][ny], or null
  // RK stage: lam_acc += a lam~, lamn = b lam~, mu = b dt lam~
  int rk;
  T a, b;
  T* lacc[3];
  int X, Y;
};

template <typename T>
__global__ void __launch_bounds__(kT) face_adj_kernel(const FaceAdjArgs<T> A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  const Geom<T>& g = A.g;
  double wsum[2] = {0.0, 0.0};
  double bsum = 0.0;
  const bool in = i < A.X && j < A.Y;
  if (in) {
    for (int c = 0; c < g.dim; ++c) {
      const int ex = g.ext(c, 0), ey = g.ext(c, 1), ez = g.ext(c, 2);
      if (i >= ex || j >= ey || k >= ez) continue;
      const int t = i + ex * (j + ey * k);
      const int p[3] = {i, j, k};
      const int ec = c == 0 ? ex : (c == 1 ? ey : ez);
      const bool boundary = !g.per[c] && (p[c] == 0 || p[c] == ec - 1);
      const T lt = adj_div_T(g, A.y, A.hy, c, i, j, k);
      const T l1 = A.lam1[c][t];
      if (A.rk) {
        // u_new = P(a u^n + b (v + dt R(v))): lam~ = P^T lam (boundary faces are imposed)
        const T lw = boundary ? T(0) : l1 + lt;
        A.lacc[c][t] += A.a * lw;
        A.lamn[c][t] = A.b * lw;
        A.mu[c][t] = A.b * A.dt * lw;
        if (c == 0 && A.bfsum && !boundary) bsum += (double)(A.b * A.dt * lw);
        continue;
      }
      if (boundary) {
        A.mu[c][t] = T(0);
        A.lamn[c][t] = T(0);
        if (c == 0 && p[0] == ec - 1 && g.bc[0][1] == FS_BC_OUTFLOW && A.lamout)
          A.lamout[j + g.ny * k] = l1 + lt;   // u^{n+1} = u* = u~ on the outflow face
        continue;
      }
      const bool forced = c < 2 && A.flags[0] && A.flags[c][t];
      T mu, direct;
      if (forced) {
        // u* = u_s, f = -R + (u_s - u)/dt, u~ = u_c on forced faces
        const T lf = A.lamf[c][t];
        mu = -lf;
        direct = -lf / A.dt;
        wsum[c] += (double)lt + (double)l1 + (double)lf / (double)A.dt;
      } else {
        const T ls = l1 + lt;
        mu = A.dt * ls;
        direct = ls;
      }
      A.mu[c][t] = mu;
      A.lamn[c][t] = direct;
      if (c == 0 && A.bfsum) bsum += (double)mu;
    }
  }
  // body-velocity adjoint sums (2-D bodies): warp reduce, one atomic per warp
  if (A.wdsum) {
    for (int c = 0; c < 2; ++c) {
      double v = wsum[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&A.wdsum[c], v);
    }
  }
  // body-force profile: the 32 threads of a warp share the row j
  if (A.bfsum) {
    double v = bsum;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && in && v != 0.0) atomicAdd(&A.bfsum[j], v);
  }
}

// Projection adjoint and stage split on grids periodic in every direction
// (uniform metrics, no body): there D^T V = -V G and the cell volume is
// constant, so P^T lam = lam - G S D lam, the forward projection.  phi = S D lam
// is solved by the forward path; this kernel forms lam~ = lam - G phi four
// cells at a time and the stage outputs lam_acc += a lam~, lam_n = b lam~
// (the predictor adjoint's mu = b dt lam~ = dt lam_n; forward Euler: a = 0,
// b = 1, no lam_acc).
template <typename T>
struct ProjAdjArgs {
  Geom<T> g;
  const T* lam[3];
  const T* phi;
  T* lacc[3];
  T* lamn[3];
  T a, b, dt;
  int rk;
  double* bfsum;
};

template <typename T>
__global__ void __launch_bounds__(kT) proj_adj4_kernel(const ProjAdjArgs<T> A) {
  const Geom<T>& g = A.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double bsum = 0.0;
  const bool in = i0 < nx && j < ny;
  if (in) {
    const size_t row = (size_t)nx * (j + (size_t)ny * k);
    const Vec4<T> p0 = ld4(A.phi + row + i0);
    const T ih[3] = {g.ihx, g.ihfy[j], g.ihz};
    for (int c = 0; c < g.dim; ++c) {
      Vec4<T> pm;
      if (c == 0) {
        const T l = __ldg(A.phi + row + (i0 > 0 ? i0 - 1 : nx - 1));
        pm = {{l, p0.v[0], p0.v[1], p0.v[2]}};
      } else if (c == 1) {
        pm = ld4(A.phi + (size_t)nx * ((j > 0 ? j - 1 : ny - 1) + (size_t)ny * k) + i0);
      } else {
        pm = ld4(A.phi + (size_t)nx * (j + (size_t)ny * (k > 0 ? k - 1 : nz - 1)) + i0);
      }
      Vec4<T> lw = ld4(A.lam[c] + row + i0);
#pragma unroll
      for (int e = 0; e < 4; ++e) lw.v[e] -= (p0.v[e] - pm.v[e]) * ih[c];
      Vec4<T> ln;
#pragma unroll
      for (int e = 0; e < 4; ++e) ln.v[e] = A.b * lw.v[e];
      if (A.rk) {
        Vec4<T> la = ld4(A.lacc[c] + row + i0);
#pragma unroll
        for (int e = 0; e < 4; ++e) la.v[e] += A.a * lw.v[e];
        st4(A.lacc[c] + row + i0, la);
      }
      st4(A.lamn[c] + row + i0, ln);
      // mu = b dt lam~ = dt lam_n is not stored: the gather transpose forms it
      if (c == 0 && A.bfsum)
        for (int e = 0; e < 4; ++e) bsum += (double)(A.dt * ln.v[e]);
    }
  }
  // body-force profile: the 32 threads of a warp share the row j
  if (A.bfsum) {
    double v = bsum;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && in && v != 0.0) atomicAdd(&A.bfsum[j], v);
  }
}

// Outflow face u*[n] = s u[n-1], s = Q_in / sum u[n-1] A: transpose into lam of u^n[n-1].
template <typename T>
__global__ void outflow_adj_kernel(const T* __restrict__ u0, const T* __restrict__ lamout, T* __restrict__ lamn0,
                                   int ex, int ny, int nz, const double* __restrict__ hy, double hz, double q_in) {
  __shared__ double s1[kT], s2[kT];
  double qo = 0.0, lu = 0.0;
  for (int t = threadIdx.x; t < ny * nz; t += blockDim.x) {
    const int j = t % ny, k = t / ny;
    const double v = (double)u0[(ex - 2) + ex * (j + ny * k)];
    qo += v * hy[j] * hz;
    lu += (double)lamout[t] * v;
  }
  s1[threadIdx.x] = qo;
  s2[threadIdx.x] = lu;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  const double Qo = s1[0], LU = s2[0];
  const double s = q_in / Qo;
  for (int t = threadIdx.x; t < ny * nz; t += blockDim.x) {
    const int j = t % ny, k = t / ny;
    const int idx = (ex - 2) + ex * (j + ny * k);
    const double area = hy[j] * hz;
    lamn0[idx] += T(s * (double)lamout[t] - s * area / Qo * LU);
  }
}

// ---- immersed boundary and body ------------------------------------------------

template <typename T>
__device__ __forceinline__ T phi_val(int kind, T r) {
  const T a = fabs(r);
  if (kind == FS_PESKIN4) {
    if (a <= T(1)) return (T(3) - T(2) * a + sqrt(fmax(T(1) + T(4) * a - T(4) * a * a, T(0)))) * T(0.125);
    if (a <= T(2)) return (T(5) - T(2) * a - sqrt(fmax(T(-7) + T(12) * a - T(4) * a * a, T(0)))) * T(0.125);
    return T(0);
  }
  if (a <= T(0.5)) return (T(1) + sqrt(fmax(T(1) - T(3) * a * a, T(0)))) / T(3);
  if (a <= T(1.5)) {
    const T b = T(1) - a;
    return (T(5) - T(3) * a - sqrt(fmax(T(1) - T(3) * b * b, T(0)))) / T(6);
  }
  return T(0);
}

// d phi / d r of the same kernels (odd in r).
template <typename T>
__device__ __forceinline__ T phi_der(int kind, T r) {
  const T a = fabs(r);
  const T sg = r < T(0) ? T(-1) : T(1);
  T d = T(0);
  if (kind == FS_PESKIN4) {
    if (a <= T(1)) {
      const T q = T(1) + T(4) * a - T(4) * a * a;
      d = (T(-2) + (q > T(0) ? (T(4) - T(8) * a) / (T(2) * sqrt(q)) : T(0))) * T(0.125);
    } else if (a <= T(2)) {
      const T q = T(-7) + T(12) * a - T(4) * a * a;
      d = (T(-2) - (q > T(0) ? (T(12) - T(8) * a) / (T(2) * sqrt(q)) : T(0))) * T(0.125);
    }
  } else {
    if (a <= T(0.5)) {
      const T q = T(1) - T(3) * a * a;
      d = (q > T(0) ? (T(-6) * a) / (T(2) * sqrt(q)) : T(0)) / T(3);
    } else if (a <= T(1.5)) {
      const T b = T(1) - a;
      const T q = T(1) - T(3) * b * b;
      // d/da of sqrt(1 - 3 (1 - a)^2) = 6 (1 - a) / (2 sqrt(q))
      d = (T(-3) - (q > T(0) ? (T(6) * b) / (T(2) * sqrt(q)) : T(0))) / T(6);
    }
  }
  return sg * d;
}

struct IBAdjGeom {
  int ex[2], ey[2];
  double x0c[2], y0c[2];
  double hx, hy;
  int kind, width;
  const double* xf;
  const double* yf;
  const double* hyv;
  const double* hfyv;
};

__device__ __forceinline__ int first_node_adj(const IBAdjGeom& G, double X, double x0, double h) {
  const double s = (X - x0) / h;
  return G.kind == FS_PESKIN4 ? (int)floor(s) - 1 : (int)floor(s + 0.5) - 1;
}
__device__ __forceinline__ double nodex(const IBAdjGeom& G, int c, int i) {
  return c == 0 ? G.xf[i] : __dmul_rn(0.5, __dadd_rn(G.xf[i], G.xf[i + 1]));
}
__device__ __forceinline__ double nodey(const IBAdjGeom& G, int c, int j) {
  return c == 1 ? G.yf[j] : __dmul_rn(0.5, __dadd_rn(G.yf[j], G.yf[j + 1]));
}

// lam_f(x) = - sum_i lam_q_i delta(x - X_i) dv(x), lam_q_i = rho dV_i lam_F (Eq. 20 transposed);
// lam_X_i = sum_c lam_q_ic sum_x f_c(x) dv(x) d delta / d r (x - X_i).
template <typename T>
__global__ void ib_force_adj_kernel(const IBAdjGeom G, int nm, const double* __restrict__ X0,
                                    const double* __restrict__ Y0, const double* __restrict__ ds,
                                    const double* __restrict__ body, const double* __restrict__ lamF, double rho,
                                    const T* __restrict__ f0, const T* __restrict__ f1, T* lf0, T* lf1,
                                    double* __restrict__ lamX) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nm) return;
  const int m = t >> 1, c = t & 1;
  const double X = X0[m] + body[0], Y = Y0[m] + body[1];
  const double lq = rho * ds[m] * G.hx * lamF[c];
  const T* f = c == 0 ? f0 : f1;
  T* lf = c == 0 ? lf0 : lf1;
  const int i0 = first_node_adj(G, X, G.x0c[c], G.hx), j0 = first_node_adj(G, Y, G.y0c[c], G.hy);
  double gx = 0.0, gy = 0.0;
  for (int b = 0; b < G.width; ++b) {
    const int j = j0 + b;
    if (j < 0 || j >= G.ey[c]) continue;
    const double ry = (nodey(G, c, j) - Y) / G.hy;
    const T py = phi_val<T>(G.kind, T(ry)), dpy = phi_der<T>(G.kind, T(ry));
    const double dvy = c == 0 ? G.hyv[j] : G.hfyv[j];
    for (int a = 0; a < G.width; ++a) {
      const int i = i0 + a;
      if (i < 0 || i >= G.ex[c]) continue;
      const double rx = (nodex(G, c, i) - X) / G.hx;
      const T px = phi_val<T>(G.kind, T(rx)), dpx = phi_der<T>(G.kind, T(rx));
      const double dv = G.hx * dvy;
      const double inv = 1.0 / (G.hx * G.hy);
      const size_t fi = (size_t)j * G.ex[c] + i;
      atomicAdd(&lf[fi], T(-lq * (double)(px * py) * inv * dv));
      const double fv = (double)f[fi] * dv;
      gx += fv * (double)(dpx * py) * inv / G.hx;
      gy += fv * (double)(px * dpy) * inv / G.hy;
    }
  }
  lamX[2 * t] = lq * gx;
  lamX[2 * t + 1] = lq * gy;
}

// Reverse of the RK4 step of Eq. (12) for one active DOF (FP64): from the adjoints
// (lw1, lv1) of (w, wdot)^{n+1} to those of (w, wdot)^n (lx0, lv0), the adjoint of the
// force lF and of the stiffness dk, linearised at the level-n state (x0, v0) and force f.
__device__ void rk4_reverse_dof(double x0, double v0, double f, double lw1, double lv1, double m, double k, double c,
                                double h, double& lx0_out, double& lv0_out, double& lF_out, double& dk_out) {
  auto acc = [&](double x, double v) { return (f - c * v - k * x) / m; };
  // forward stages
  const double k1x = v0, k1v = acc(x0, v0);
  const double x1 = x0 + 0.5 * h * k1x, v1 = v0 + 0.5 * h * k1v;
  const double k2x = v1, k2v = acc(x1, v1);
  const double x2 = x0 + 0.5 * h * k2x, v2 = v0 + 0.5 * h * k2v;
  const double k3x = v2;
  const double x3 = x0 + h * k3x;
  double lF = 0.0, dk = 0.0;
  // reverse
  double lx0 = lw1, lv0 = lv1;
  double lk1x = h / 6.0 * lw1, lk2x = h / 3.0 * lw1, lk3x = h / 3.0 * lw1, lk4x = h / 6.0 * lw1;
  double lk1v = h / 6.0 * lv1, lk2v = h / 3.0 * lv1, lk3v = h / 3.0 * lv1, lk4v = h / 6.0 * lv1;
  // k4v = acc(x3, v3), k4x = v3
  double lx3 = -k / m * lk4v, lv3 = -c / m * lk4v + lk4x;
  lF += lk4v / m;
  dk += -x3 / m * lk4v;
  lx0 += lx3;
  lk3x += h * lx3;
  lv0 += lv3;
  lk3v += h * lv3;
  // k3v = acc(x2, v2), k3x = v2
  double lx2 = -k / m * lk3v, lv2 = -c / m * lk3v + lk3x;
  lF += lk3v / m;
  dk += -x2 / m * lk3v;
  lx0 += lx2;
  lk2x += 0.5 * h * lx2;
  lv0 += lv2;
  lk2v += 0.5 * h * lv2;
  // k2v = acc(x1, v1), k2x = v1
  double lx1 = -k / m * lk2v, lv1s = -c / m * lk2v + lk2x;
  lF += lk2v / m;
  dk += -x1 / m * lk2v;
  lx0 += lx1;
  lk1x += 0.5 * h * lx1;
  lv0 += lv1s;
  lk1v += 0.5 * h * lv1s;
  // k1v = acc(x0, v0), k1x = v0
  lx0 += -k / m * lk1v;
  lv0 += -c / m * lk1v + lk1x;
  lF += lk1v / m;
  dk += -x0 / m * lk1v;
  lx0_out = lx0;
  lv0_out = lv0;
  lF_out = lF;
  dk_out = dk;
}

// Reverse of the RK4 step of Eq. (12) per active DOF; body state and adjoints in FP64.
//   lamb:  in lam of (w, wdot)^{n+1}, out: lam of (w, wdot)^n from the ODE
//   lamF:  out lam of F^n (plus the direct dJ/dF)
__global__ void rk4_adj_kernel(const double* __restrict__ st, const double* __restrict__ F, double* __restrict__ lamb,
                               double* __restrict__ lamF, const double* __restrict__ dJdF, double m, double k,
                               double c, int ax, int ay, double dt, int dynamic, double* __restrict__ gk) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int act[2] = {ax, ay};
  double dk = 0.0;
  for (int d = 0; d < 2; ++d) {
    const double lw1 = lamb[d], lv1 = lamb[2 + d];
    const double lF = dJdF[d];
    if (!dynamic) {   // static body: state carried through unchanged
      lamF[d] = lF;
      continue;
    }
    if (!act[d]) {
      lamb[d] = 0.0;
      lamb[2 + d] = 0.0;
      lamF[d] = lF;
      continue;
    }
    double lx0, lv0, lFo, dkd;
    rk4_reverse_dof(st[d], st[2 + d], F[d], lw1, lv1, m, k, c, dt, lx0, lv0, lFo, dkd);
    lamb[d] = lx0;
    lamb[2 + d] = lv0;
    lamF[d] = lF + lFo;
    dk += dkd;
  }
  if (gk) *gk += dk;
}

// Implicit-differentiation solve of the strongly coupled step (§2.4.1, the
// fixed point s* = B(s^n, F(u^n, s*), k) of Algorithm 1), one thread, FP64.
//   sig    lam of the step's output body state s* (the caller's lam->body)
//   base   the fluid adjoint's body part for the loss seeds: U_s^T lam_u + J_s^T dJdF
//   unit   the fluid adjoint's body part for a unit force adjoint e_d: J_s^T e_d (4 per DOF)
// Forms dB/ds* = B_F J_s (B_F^T from the RK4 reverse of unit adjoints), solves
// (I - dB/ds*)^T mu = sig + base by Gaussian elimination with partial pivoting,
// and writes lam of s^n = B_s^T mu into lamb, beta = B_F^T mu (the force adjoint the
// fluid solves add on top of dJdF) and dJ/dk += B_k^T mu.
__global__ void coupled_adj_solve_kernel(const double* __restrict__ s_n, const double* __restrict__ F,
                                         const double* __restrict__ sig, const double* __restrict__ base,
                                         const double* __restrict__ unit, double m, double k, double c, int ax,
                                         int ay, double dt, double* __restrict__ lamb, double* __restrict__ beta,
                                         double* __restrict__ gk, int* __restrict__ singular) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int act[2] = {ax, ay};
  double BFt[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};   // (B_F^T e_j)_d
  double Bst[4][4] = {};                              // column j: B_s^T e_j
  double Bk[4] = {0, 0, 0, 0};
  for (int j = 0; j < 4; ++j)
    for (int d = 0; d < 2; ++d) {
      if (!act[d]) continue;
      const double lw1 = j == d ? 1.0 : 0.0, lv1 = j == 2 + d ? 1.0 : 0.0;
      if (lw1 == 0.0 && lv1 == 0.0) continue;
      double lx0, lv0, lF, dk;
      rk4_reverse_dof(s_n[d], s_n[2 + d], F[d], lw1, lv1, m, k, c, dt, lx0, lv0, lF, dk);
      BFt[d][j] = lF;
      Bst[d][j] = lx0;
      Bst[2 + d][j] = lv0;
      Bk[j] = dk;
    }
  // A = (I - dB/ds*)^T = I - M, M[i][j] = sum_d unit_d[i] BFt[d][j]
  double A[4][5];
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) {
      double mij = 0.0;
      for (int d = 0; d < 2; ++d)
        if (act[d]) mij += unit[4 * d + i] * BFt[d][j];
      A[i][j] = (i == j ? 1.0 : 0.0) - mij;
    }
    A[i][4] = sig[i] + base[i];
  }
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (!(fabs(A[piv][col]) > 0.0)) {
      *singular = 1;
      return;
    }
    if (piv != col)
      for (int q = 0; q < 5; ++q) {
        const double t = A[col][q];
        A[col][q] = A[piv][q];
        A[piv][q] = t;
      }
    for (int r = col + 1; r < 4; ++r) {
      const double f = A[r][col] / A[col][col];
      for (int q = col; q < 5; ++q) A[r][q] -= f * A[col][q];
    }
  }
  double mu[4];
  for (int i = 3; i >= 0; --i) {
    double r = A[i][4];
    for (int q = i + 1; q < 4; ++q) r -= A[i][q] * mu[q];
    mu[i] = r / A[i][i];
  }
  double dk = 0.0;
  for (int i = 0; i < 4; ++i) {
    double r = 0.0;
    for (int j = 0; j < 4; ++j) r += Bst[i][j] * mu[j];
    lamb[i] = r;
    dk += Bk[i] * mu[i];
  }
  for (int d = 0; d < 2; ++d) {
    double r = 0.0;
    for (int j = 0; j < 4; ++j) r += BFt[d][j] * mu[j];
    beta[d] = r;
  }
  if (gk) *gk += dk;
  *singular = 0;
}

// y += (*alpha) x (alpha read on the device)
template <typename T>
__global__ void axpy_dev_kernel(T* __restrict__ y, const T* __restrict__ x, const double* __restrict__ alpha,
                                long long n) {
  const T a = T(*alpha);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] += a * x[t];
}

// lam of (w, wdot)^n += position adjoint (sum over markers) + fluid sums of the body velocity.
__global__ void body_adj_finish_kernel(int nm, const double* __restrict__ lamX, const double* __restrict__ wdsum,
                                       double* __restrict__ lamb) {
  __shared__ double sx[kT], sy[kT];
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < 2 * nm; t += blockDim.x) {
    a += lamX[2 * t];
    b += lamX[2 * t + 1];
  }
  sx[threadIdx.x] = a;
  sy[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sx[threadIdx.x] += sx[threadIdx.x + o];
      sy[threadIdx.x] += sy[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    lamb[0] += sx[0];
    lamb[1] += sy[0];
    lamb[2] += wdsum[0];
    lamb[3] += wdsum[1];
  }
}

template <typename T>
__global__ void axpy_kernel(T* __restrict__ y, const T* __restrict__ x, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] += x[t];
}

IBAdjGeom make_ib_adj_geom(const fs_grid* G) {
  IBAdjGeom g;
  for (int c = 0; c < 2; ++c) {
    g.ex[c] = G->nx + ((c == 0 && !G->per[0]) ? 1 : 0);
    g.ey[c] = G->ny + ((c == 1 && !G->per[1]) ? 1 : 0);
  }
  g.hx = G->hx;
  g.hy = G->h[1][0];
  g.x0c[0] = G->xf[0][0];
  g.x0c[1] = 0.5 * (G->xf[0][0] + G->xf[0][1]);
  g.y0c[0] = 0.5 * (G->xf[1][0] + G->xf[1][1]);
  g.y0c[1] = G->xf[1][0];
  g.kind = G->ib.kernel;
  g.width = G->ib.kernel == FS_PESKIN4 ? 4 : 3;
  g.xf = G->xf64[0];
  g.yf = G->xf64[1];
  g.hyv = G->hy64;
  g.hfyv = G->hfy64;
  return g;
}

size_t comp_count(const fs_grid* G, int c) {
  size_t s = 1;
  const int n[3] = {G->nx, G->ny, G->nz};
  for (int d = 0; d < 3; ++d) s *= (size_t)(n[d] + ((c == d && !G->per[d]) ? 1 : 0));
  return s;
}

template <typename T>
void launch_rhs_adjoint(fs_grid* G, T* const* u, T* const* mu, T* const* lam) {
  RhsAdjArgs<T> A;
  A.g = G->geom<T>();
  for (int c = 0; c < 3; ++c) {
    A.u[c] = c < G->dim ? u[c] : nullptr;
    A.mu[c] = c < G->dim ? mu[c] : nullptr;
    A.lam[c] = c < G->dim ? lam[c] : nullptr;
  }
  A.conv = G->conv;
  A.X = G->nx + (G->per[0] ? 0 : 1);
  A.Y = G->ny + (G->per[1] ? 0 : 1);
  const dim3 blk = stencil_block(G), grd = stencil_grid(G, A.X, A.Y);
  FS_LAUNCH(G, "rhs_adjoint", rhs_adjoint_kernel<T><<<grd, blk, 0, G->stream>>>(A));
}

// adjoint Poisson: spec = S (V^-1 (-G^T lam))
template <typename T>
void launch_projection_adjoint_solve(fs_grid* G, T* const* lam, T* spec) {
  const Geom<T> g = G->geom<T>();
  const dim3 blk = stencil_block(G), grd = stencil_grid(G, G->nx, G->ny);
  FS_LAUNCH(G, "adj_rhs", adj_rhs_kernel<T><<<grd, blk, 0, G->stream>>>(g, lam[0], lam[1], G->dim == 3 ? lam[2] : lam[1],
                                                                        G->hy64, spec));
  // the adjoint uses the solution through its gradient and D^T (boundary faces are imposed), so
  // the zero mode's gauge is not set
  G->ygauge = false;
  poisson_solve_inplace<T>(G, spec);
  G->ygauge = true;
}

// Fully periodic 3-D grids with central convection and no body: the gather
// transpose of the flux stencil applies.
bool gather_fast(const fs_grid* G) {
  return G->dim == 3 && G->per[0] && G->per[1] && G->per[2] && G->conv == FS_CENTRAL2 && !G->has_body;
}

// True when the projection adjoint may take the forward projection (all
// directions periodic, no body, four-cell rows on 16/32-byte aligned arrays).
template <typename T>
bool proj_adj_fast(const fs_grid* G, T* const* lam, T* const* la, T* const* ln) {
  if (G->has_body || G->nx % 4) return false;
  for (int d = 0; d < G->dim; ++d)
    if (!G->per[d]) return false;
  const uintptr_t al = 4 * sizeof(T);
  if ((uintptr_t)G->spec % al) return false;
  for (int c = 0; c < G->dim; ++c)
    if ((uintptr_t)lam[c] % al || (uintptr_t)la[c] % al || (uintptr_t)ln[c] % al) return false;
  return true;
}

template <typename T>
void launch_proj_adj_fast(fs_grid* G, T* const* lam, double a, double b, double dt, bool rk, double* bfsum,
                          T* const* la, T* const* ln) {
  T* spec = (T*)G->spec;
  G->ygauge = false;   // only the gradient of the solution is used
  poisson_solve_from_velocity<T>(G, make_div_args<T>(G, lam, nullptr), spec);
  G->ygauge = true;
  ProjAdjArgs<T> A;
  A.g = G->geom<T>();
  for (int c = 0; c < 3; ++c) {
    const bool on = c < G->dim;
    A.lam[c] = on ? lam[c] : nullptr;
    A.lacc[c] = on ? la[c] : nullptr;
    A.lamn[c] = on ? ln[c] : nullptr;
  }
  A.phi = spec;
  A.a = (T)a;
  A.b = (T)b;
  A.dt = (T)dt;
  A.rk = rk ? 1 : 0;
  A.bfsum = bfsum;
  const dim3 blk(32, 8), grd((G->nx / 4 + 31) / 32, (G->ny + 7) / 8, G->nz);
  FS_LAUNCH(G, "proj_adjoint", proj_adj4_kernel<T><<<grd, blk, 0, G->stream>>>(A));
}

// out = src + R'(u)^T (scale src) on a fully periodic grid (gather transpose).
template <typename T>
void launch_rhs_adjoint_gather(fs_grid* G, T* const* u, T* const* src, double scale, T* const* out,
                               T* const* add = nullptr) {
  GatherAdjArgs<T> A;
  A.r.g = G->geom<T>();
  for (int c = 0; c < 3; ++c) {
    A.r.u[c] = u[c];
    A.r.mu[c] = src[c];
    A.r.lam[c] = nullptr;
    A.out[c] = out[c];
    A.add[c] = add ? add[c] : nullptr;
  }
  A.r.conv = G->conv;
  A.r.X = G->nx;
  A.r.Y = G->ny;
  A.scale = (T)scale;
  if constexpr (std::is_same<T, float>::value) {
    bool vec = G->nx % 4 == 0;
    for (int c = 0; c < 3; ++c)
      vec = vec && (uintptr_t)u[c] % 16 == 0 && (uintptr_t)src[c] % 16 == 0 && (uintptr_t)out[c] % 16 == 0 &&
          (!add || (uintptr_t)add[c] % 16 == 0);
    if (vec) {
      const dim3 vb(32, 8), vg((G->nx / 4 + 31) / 32, (G->ny + 7) / 8, G->nz);
      FS_LAUNCH(G, "rhs_adjoint", rhs_adjoint_gather4_kernel<<<vg, vb, 0, G->stream>>>(A));
      return;
    }
  }
  const dim3 blk = stencil_block(G), grd = stencil_grid(G, G->nx, G->ny);
  FS_LAUNCH(G, "rhs_adjoint", rhs_adjoint_gather_kernel<T><<<grd, blk, 0, G->stream>>>(A));
}

}  // namespace

// Adjoint work buffers (allocated on the first adjoint call of a grid).
struct AdjBuffers {
  void* mu[3] = {nullptr, nullptr, nullptr};
  void* lamn[3] = {nullptr, nullptr, nullptr};
  void* lacc[3] = {nullptr, nullptr, nullptr};
  void* v1[3] = {nullptr, nullptr, nullptr};
  void* v2[3] = {nullptr, nullptr, nullptr};
  void* lamf[2] = {nullptr, nullptr};
  void* lamout = nullptr;
  double* scal = nullptr;   // [0..1] lamF, [2..3] wdsum, [4..5] dJdF, [8..] lamX (2 * 2 * nm)
  // strongly coupled steps: a copy of the state for the forward re-run, the fluid
  // adjoint of a unit force adjoint per DOF, and the small FP64 work vectors
  void* cu[3] = {nullptr, nullptr, nullptr};
  void* ld[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  double* cd = nullptr;
};

int adj_buffers(fs_grid* G, AdjBuffers** out) {
  if (G->adj) {
    *out = (AdjBuffers*)G->adj;
    return FS_OK;
  }
  AdjBuffers* B = new AdjBuffers();
  const size_t es = G->prec == FS_MIXED ? 4 : 8;
  bool ok = true;
  for (int c = 0; c < G->dim && ok; ++c) {
    const size_t n = comp_count(G, c) * es;
    ok = cudaMalloc(&B->mu[c], n) == cudaSuccess && cudaMalloc(&B->lamn[c], n) == cudaSuccess &&
         cudaMalloc(&B->lacc[c], n) == cudaSuccess;
    if (ok && G->scheme == FS_RK3)
      ok = cudaMalloc(&B->v1[c], n) == cudaSuccess && cudaMalloc(&B->v2[c], n) == cudaSuccess;
  }
  if (ok && G->has_body)
    for (int c = 0; c < 2 && ok; ++c) ok = cudaMalloc(&B->lamf[c], comp_count(G, c) * es) == cudaSuccess;
  if (ok) ok = cudaMalloc(&B->lamout, (size_t)G->ny * G->nz * es) == cudaSuccess;
  const size_t ns = 16 + 4 * (size_t)(G->has_body ? G->ib.nm : 0);
  if (ok) ok = cudaMalloc(&B->scal, ns * sizeof(double)) == cudaSuccess;
  if (!ok) {
    free_adj_buffers(B);
    return set_error(FS_ERR_CUDA, "allocating adjoint buffers");
  }
  G->adj = B;
  *out = B;
  return FS_OK;
}

void free_adj_buffers(void* p) {
  AdjBuffers* B = (AdjBuffers*)p;
  if (!B) return;
  auto F = [](void* q) {
    if (q) cudaFree(q);
  };
  for (int c = 0; c < 3; ++c) {
    F(B->mu[c]);
    F(B->lamn[c]);
    F(B->lacc[c]);
    F(B->v1[c]);
    F(B->v2[c]);
  }
  F(B->lamf[0]);
  F(B->lamf[1]);
  F(B->lamout);
  F(B->scal);
  for (int c = 0; c < 3; ++c) {
    F(B->cu[c]);
    F(B->ld[0][c]);
    F(B->ld[1][c]);
  }
  F(B->cd);
  delete B;
}

int coupled_buffers(fs_grid* G, AdjBuffers* B) {
  if (B->cd) return FS_OK;
  const size_t es = G->prec == FS_MIXED ? 4 : 8;
  bool ok = true;
  for (int c = 0; c < G->dim && ok; ++c) {
    const size_t n = comp_count(G, c) * es;
    ok = cudaMalloc(&B->cu[c], n) == cudaSuccess && cudaMalloc(&B->ld[0][c], n) == cudaSuccess &&
         cudaMalloc(&B->ld[1][c], n) == cudaSuccess;
  }
  if (ok) ok = cudaMalloc(&B->cd, 32 * sizeof(double)) == cudaSuccess;
  if (!ok) return set_error(FS_ERR_CUDA, "allocating the coupled adjoint buffers");
  return FS_OK;
}

// Recompute the forward-Euler step's classification, u*, forcing f and force F from
// the velocity u and the body kinematics s_lin (the point the adjoint is linearised at).
template <typename T>
void fe_body_recompute(fs_grid* G, T* const* u, double* s_lin, double dt) {
  T* us[3] = {(T*)G->ustar[0], (T*)G->ustar[1], (T*)G->ustar[2]};
  ib_prepare<T>(G, s_lin);
  launch_outflow_flux<T>(G, u);
  launch_predictor<T>(G, u, nullptr, us, dt, 0.0, 1.0, s_lin);
  ib_forces<T>(G, s_lin);
}

// Fluid part of the forward-Euler adjoint: lam of u^{n+1} in L is overwritten with
// lam of u^n.  With a body (s_lin not null; the forward quantities recomputed at
// s_lin by fe_body_recompute), lamF (device, 2) is the adjoint of the step's force,
// spread back to the forcing term (Eq. 20 transposed), and lamb (device, 4) receives
// the fluid's dependence on the body kinematics: the marker-position adjoint and the
// adjoint of the body velocity imposed on forced faces.
template <typename T>
void fe_fluid_adjoint(fs_grid* G, AdjBuffers* B, T* const* u, const double* s_lin, T* const* L, const double* lamF,
                      double* lamb, double* bfsum, double dt) {
  const Geom<T> g = G->geom<T>();
  const int X = G->nx + (G->per[0] ? 0 : 1), Y = G->ny + (G->per[1] ? 0 : 1);
  const dim3 blk = stencil_block(G), grd = stencil_grid(G, X, Y);
  T* mu[3] = {(T*)B->mu[0], (T*)B->mu[1], (T*)B->mu[2]};
  T* ln[3] = {(T*)B->lamn[0], (T*)B->lamn[1], (T*)B->lamn[2]};
  T* spec = (T*)G->spec;
  IBDev& ib = G->ib;
  double* sc = B->scal;
  const bool body = s_lin != nullptr;
  if (body) {
    for (int c = 0; c < 2; ++c) cudaMemsetAsync(B->lamf[c], 0, comp_count(G, c) * sizeof(T), G->stream);
    cudaMemsetAsync(sc + 2, 0, 2 * sizeof(double), G->stream);
    // force reverse: lam_f on the grid, marker position adjoint
    const IBAdjGeom ig = make_ib_adj_geom(G);
    FS_LAUNCH(G, "ib_force_adjoint", ib_force_adj_kernel<T><<<(2 * ib.nm + 127) / 128, 128, 0, G->stream>>>(
                                         ig, ib.nm, ib.X0, ib.Y0, ib.ds, s_lin, lamF, G->rho, (const T*)ib.f[0],
                                         (const T*)ib.f[1], (T*)B->lamf[0], (T*)B->lamf[1], sc + 8));
  }
  launch_projection_adjoint_solve<T>(G, L, spec);
  FaceAdjArgs<T> A{};
  A.g = g;
  for (int c = 0; c < 3; ++c) {
    A.lam1[c] = L[c];
    A.mu[c] = mu[c];
    A.lamn[c] = ln[c];
  }
  A.y = spec;
  A.hy = G->hy64;
  A.dt = (T)dt;
  A.rk = 0;
  if (body) {
    A.flags[0] = ib.flags[0];
    A.flags[1] = ib.flags[1];
    A.lamf[0] = (const T*)B->lamf[0];
    A.lamf[1] = (const T*)B->lamf[1];
    A.wdsum = sc + 2;
  }
  A.bfsum = bfsum;
  A.lamout = (T*)B->lamout;
  A.X = X;
  A.Y = Y;
  FS_LAUNCH(G, "face_adjoint", face_adj_kernel<T><<<grd, blk, 0, G->stream>>>(A));
  launch_rhs_adjoint<T>(G, u, mu, ln);
  if (!G->per[0] && G->bc[0][1] == FS_BC_OUTFLOW) {
    double q_in = 0.0;
    if (G->bc[0][0] == FS_BC_INFLOW) {
      double area = 0.0;
      for (int j = 0; j < G->ny; ++j) area += G->h[1][j];
      area *= (G->dim == 3 ? G->hz * G->nz : 1.0);
      q_in = G->bcv[0][0][0] * area;
    }
    FS_LAUNCH(G, "outflow_adjoint", outflow_adj_kernel<T><<<1, kT, 0, G->stream>>>(
                                        u[0], (const T*)B->lamout, ln[0], G->nx + 1, G->ny, G->nz, G->hy64,
                                        G->dim == 3 ? G->hz : 1.0, q_in));
  }
  if (body)
    FS_LAUNCH(G, "body_adjoint", body_adj_finish_kernel<<<1, kT, 0, G->stream>>>(ib.nm, sc + 8, sc + 2, lamb));
  for (int c = 0; c < G->dim; ++c)
    cudaMemcpyAsync(L[c], ln[c], comp_count(G, c) * sizeof(T), cudaMemcpyDeviceToDevice, G->stream);
}

template <typename T>
int step_adjoint(fs_grid* G, const fs_state* st, fs_state* lam, const double* dJdF, fs_param_grad* pg, double dt,
                 void* const* rv1, void* const* rv2, bool dJdF_on_device) {
  AdjBuffers* B = nullptr;
  int rc = adj_buffers(G, &B);
  if (rc != FS_OK) return rc;
  const int dim = G->dim;
  T* u[3] = {(T*)st->u[0], (T*)st->u[1], (T*)(dim == 3 ? st->u[2] : nullptr)};
  T* L[3] = {(T*)lam->u[0], (T*)lam->u[1], (T*)(dim == 3 ? lam->u[2] : nullptr)};
  T* mu[3] = {(T*)B->mu[0], (T*)B->mu[1], (T*)B->mu[2]};
  T* ln[3] = {(T*)B->lamn[0], (T*)B->lamn[1], (T*)B->lamn[2]};
  T* la[3] = {(T*)B->lacc[0], (T*)B->lacc[1], (T*)B->lacc[2]};
  T* spec = (T*)G->spec;
  const Geom<T> g = G->geom<T>();
  const int X = G->nx + (G->per[0] ? 0 : 1), Y = G->ny + (G->per[1] ? 0 : 1);
  const dim3 blk = stencil_block(G), grd = stencil_grid(G, X, Y);
  double* bfsum = pg ? pg->body_force : nullptr;

  if (G->scheme == FS_RK3) {
    // the stage states v1, v2 of the forward step: recorded by it, or recomputed here
    T* us[3] = {(T*)G->ustar[0], (T*)G->ustar[1], (T*)G->ustar[2]};
    T* v1[3] = {(T*)B->v1[0], (T*)B->v1[1], (T*)B->v1[2]};
    T* v2[3] = {(T*)B->v2[0], (T*)B->v2[1], (T*)B->v2[2]};
    const double Ac[3] = {0.0, 0.75, 1.0 / 3.0}, Bc[3] = {1.0, 0.25, 2.0 / 3.0};
    if (rv1 && rv2) {
      for (int c = 0; c < 3; ++c) {
        v1[c] = c < dim ? (T*)rv1[c] : nullptr;
        v2[c] = c < dim ? (T*)rv2[c] : nullptr;
      }
    } else {
      // as the forward step took them (its stage solves leave the pressure's gauge unset)
      G->ygauge = false;
      launch_predictor<T>(G, u, u, us, dt, Ac[0], Bc[0], nullptr);
      poisson_solve_from_velocity<T>(G, make_div_args<T>(G, us, nullptr), spec);
      launch_correct<T>(G, us, spec, v1);
      launch_predictor<T>(G, v1, u, us, dt, Ac[1], Bc[1], nullptr);
      poisson_solve_from_velocity<T>(G, make_div_args<T>(G, us, nullptr), spec);
      launch_correct<T>(G, us, spec, v2);
      G->ygauge = true;
    }
    T* const* vs[3] = {u, v1, v2};
    for (int c = 0; c < dim; ++c) cudaMemsetAsync(la[c], 0, comp_count(G, c) * sizeof(T), G->stream);
    // cur = lam of the stage output, starting from lam^{n+1}
    T* cur[3] = {L[0], L[1], L[2]};
    const bool fast = gather_fast(G) && proj_adj_fast<T>(G, L, la, ln);
    if (fast) {
      // lam of v_s = b lam~ + R'(v_s)^T (b dt lam~), written straight into lam->u
      // (the last stage's gather also adds the stage accumulator: lam^n = lam of v_0 + lam_acc)
      for (int s = 2; s >= 0; --s) {
        launch_proj_adj_fast<T>(G, L, Ac[s], Bc[s], dt, true, bfsum, la, ln);
        launch_rhs_adjoint_gather<T>(G, vs[s], ln, dt, L, s == 0 ? la : nullptr);
      }
      return cuda_check(cudaGetLastError(), "fs_step_adjoint (RK3)");
    }
    for (int s = 2; s >= 0; --s) {
      launch_projection_adjoint_solve<T>(G, cur, spec);
      FaceAdjArgs<T> A{};
      A.g = g;
      for (int c = 0; c < 3; ++c) {
        A.lam1[c] = cur[c];
        A.mu[c] = mu[c];
        A.lamn[c] = ln[c];
        A.lacc[c] = la[c];
      }
      A.y = spec;
      A.hy = G->hy64;
      A.dt = (T)dt;
      A.rk = 1;
      A.a = (T)Ac[s];
      A.b = (T)Bc[s];
      A.bfsum = bfsum;
      A.X = X;
      A.Y = Y;
      FS_LAUNCH(G, "face_adjoint", face_adj_kernel<T><<<grd, blk, 0, G->stream>>>(A));
      // lam of v_s = b lam~ + R'(v_s)^T (b dt lam~)
      launch_rhs_adjoint<T>(G, vs[s], mu, ln);
      if (s > 0) {
        for (int c = 0; c < dim; ++c) {
          // the next stage reads cur; stage s-1 output adjoint becomes ln: swap buffers through lam->u
          cudaMemcpyAsync(L[c], ln[c], comp_count(G, c) * sizeof(T), cudaMemcpyDeviceToDevice, G->stream);
          cur[c] = L[c];
        }
      }
    }
    // lam^n = lam_acc + lam of v_0 (= u^n)
    for (int c = 0; c < dim; ++c) {
      const long long n = (long long)comp_count(G, c);
      FS_LAUNCH(G, "axpy", axpy_kernel<T><<<(int)std::min<long long>((n + 255) / 256, 148 * 16), 256, 0,
                                          G->stream>>>(la[c], ln[c], n));
      cudaMemcpyAsync(L[c], la[c], n * sizeof(T), cudaMemcpyDeviceToDevice, G->stream);
    }
    return cuda_check(cudaGetLastError(), "fs_step_adjoint (RK3)");
  }

  // ---- forward Euler (optional body) ------------------------------------------
  IBDev& ib = G->ib;
  double* sc = B->scal;
  if (G->has_body) {
    // recompute the classification, u*, f and F of the forward step from the state at n
    fe_body_recompute<T>(G, u, st->body, dt);
    if (dJdF_on_device) {
      if (dJdF) cudaMemcpyAsync(sc + 4, dJdF, 2 * sizeof(double), cudaMemcpyDeviceToDevice, G->stream);
      else cudaMemsetAsync(sc + 4, 0, 2 * sizeof(double), G->stream);
    } else {
      double h4[2] = {dJdF ? dJdF[0] : 0.0, dJdF ? dJdF[1] : 0.0};
      cudaMemcpyAsync(sc + 4, h4, 2 * sizeof(double), cudaMemcpyHostToDevice, G->stream);
    }
    // body ODE reverse: lam of (w, wdot)^{n+1} -> ODE part of lam^n, lam_F, dJ/dk
    FS_LAUNCH(G, "rk4_adjoint", rk4_adj_kernel<<<1, 32, 0, G->stream>>>(
                                    st->body, ib.F, lam->body, sc, sc + 4, ib.mass, ib.k, ib.c, ib.active[0],
                                    ib.active[1], dt, ib.mass > 0 ? 1 : 0, pg ? pg->stiffness : nullptr));
    fe_fluid_adjoint<T>(G, B, u, st->body, L, sc, lam->body, bfsum, dt);
    return cuda_check(cudaGetLastError(), "fs_step_adjoint");
  }
  if (G->bc[0][1] == FS_BC_OUTFLOW && !G->per[0]) {
    launch_outflow_flux<T>(G, u);
  } else if (gather_fast(G) && proj_adj_fast<T>(G, L, la, ln)) {
    launch_proj_adj_fast<T>(G, L, 0.0, 1.0, dt, false, bfsum, la, ln);
    launch_rhs_adjoint_gather<T>(G, u, ln, dt, L);
    return cuda_check(cudaGetLastError(), "fs_step_adjoint");
  }
  fe_fluid_adjoint<T>(G, B, u, nullptr, L, nullptr, nullptr, bfsum, dt);
  return cuda_check(cudaGetLastError(), "fs_step_adjoint");
}

// Adjoint of the strongly coupled forward-Euler FSI step (§2.3.3 Algorithm 1,
// differentiated implicitly as in §2.4.1).  The forward sub-iteration is re-run
// from st_n to its converged body state s*; the fluid step is linearised at
// (u^n, s*) and the body step at (s^n, F(u^n, s*)).  With U the fluid's new
// velocity, F its force, B the RK4 step and J_s, J_u the force's partial
// derivatives:
//   mu solves (I - B_F J_s)^T mu = lam_s + U_s^T lam_u + J_s^T dJdF,
//   lam_u^n = U_u^T lam_u + J_u^T (dJdF + B_F^T mu),  lam_s^n = B_s^T mu,
//   dJ/dk += B_k^T mu.
// The fluid adjoint is run once for the loss seeds and once per active DOF for a
// unit force adjoint (J_u^T e_d, J_s^T e_d); the 4 x 4 system is solved on the device.
template <typename T>
int step_adjoint_coupled(fs_grid* G, const fs_state* st, fs_state* lam, const double* dJdF, bool dJdF_on_device,
                         fs_param_grad* pg, double dt) {
  AdjBuffers* B = nullptr;
  int rc = adj_buffers(G, &B);
  if (rc != FS_OK) return rc;
  rc = coupled_buffers(G, B);
  if (rc != FS_OK) return rc;
  if (pg && pg->body_force)
    return set_error(FS_ERR_UNSUPPORTED, "body-force gradient of a strongly coupled FSI step");
  IBDev& ib = G->ib;
  cudaStream_t s = G->stream;
  const int dim = G->dim;
  T* u[3] = {(T*)st->u[0], (T*)st->u[1], nullptr};
  T* L[3] = {(T*)lam->u[0], (T*)lam->u[1], nullptr};
  double* d = B->cd;
  double* s_star = d;          // [0..3]
  double* sig = d + 4;         // [4..7]
  double* base = d + 8;        // [8..11]
  double* unit = d + 12;       // [12..19], 4 per DOF
  double* fbar = d + 20;       // [20..21]
  double* e = d + 22;          // [22..25] unit force adjoints e_0, e_1
  double* beta = d + 26;       // [26..27]
  int* singular = (int*)(d + 28);
  // 1. the converged body state of the forward step, from copies of st_n
  for (int c = 0; c < dim; ++c)
    cudaMemcpyAsync(B->cu[c], st->u[c], comp_count(G, c) * sizeof(T), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(s_star, st->body, 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  fs_state tmp{};
  for (int c = 0; c < dim; ++c) tmp.u[c] = B->cu[c];
  tmp.body = s_star;
  const int iters = G->fsi_last_iters;
  const double xi = G->fsi_last_xi;
  rc = step_coupled<T>(G, &tmp, dt, false);
  G->fsi_last_iters = iters;
  G->fsi_last_xi = xi;
  if (rc != FS_OK) return rc;
  // 2. the fluid step at (u^n, s*): classification, u*, f and F*
  fe_body_recompute<T>(G, u, s_star, dt);
  // 3. seeds
  cudaMemcpyAsync(sig, lam->body, 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (dJdF_on_device) {
    if (dJdF) cudaMemcpyAsync(fbar, dJdF, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    else cudaMemsetAsync(fbar, 0, 2 * sizeof(double), s);
  } else {
    const double h2[2] = {dJdF ? dJdF[0] : 0.0, dJdF ? dJdF[1] : 0.0};
    cudaMemcpyAsync(fbar, h2, 2 * sizeof(double), cudaMemcpyHostToDevice, s);
  }
  const double he[4] = {1.0, 0.0, 0.0, 1.0};
  cudaMemcpyAsync(e, he, 4 * sizeof(double), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(base, 0, 12 * sizeof(double), s);
  // 4. fluid adjoints: the loss seeds, then a unit force adjoint per active DOF
  fe_fluid_adjoint<T>(G, B, u, s_star, L, fbar, base, nullptr, dt);
  for (int q = 0; q < 2; ++q) {
    if (!ib.active[q]) continue;
    T* Lq[3] = {(T*)B->ld[q][0], (T*)B->ld[q][1], nullptr};
    for (int c = 0; c < dim; ++c) cudaMemsetAsync(Lq[c], 0, comp_count(G, c) * sizeof(T), s);
    fe_fluid_adjoint<T>(G, B, u, s_star, Lq, e + 2 * q, unit + 4 * q, nullptr, dt);
  }
  // 5. the implicit system, then lam_u^n += beta_d J_u^T e_d
  FS_LAUNCH(G, "coupled_adjoint_solve", coupled_adj_solve_kernel<<<1, 32, 0, s>>>(
                                            st->body, ib.F, sig, base, unit, ib.mass, ib.k, ib.c, ib.active[0],
                                            ib.active[1], dt, lam->body, beta, pg ? pg->stiffness : nullptr,
                                            singular));
  for (int q = 0; q < 2; ++q) {
    if (!ib.active[q]) continue;
    for (int c = 0; c < dim; ++c) {
      const long long n = (long long)comp_count(G, c);
      FS_LAUNCH(G, "axpy", axpy_dev_kernel<T><<<(int)std::min<long long>((n + 255) / 256, 148 * 16), 256, 0, s>>>(
                               L[c], (const T*)B->ld[q][c], beta + q, n));
    }
  }
  int hs = 0;
  cudaError_t err = cudaMemcpyAsync(&hs, singular, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_check(err, "fs_step_adjoint (strong coupling)");
  if (hs) return set_error(FS_ERR_DIVERGED, "fs_step_adjoint: singular coupling system (I - dB/ds)");
  return cuda_check(cudaGetLastError(), "fs_step_adjoint (strong coupling)");
}

template int step_adjoint<float>(fs_grid*, const fs_state*, fs_state*, const double*, fs_param_grad*, double,
                                  void* const*, void* const*, bool);
template int step_adjoint<double>(fs_grid*, const fs_state*, fs_state*, const double*, fs_param_grad*, double,
                                   void* const*, void* const*, bool);
template int step_adjoint_coupled<float>(fs_grid*, const fs_state*, fs_state*, const double*, bool, fs_param_grad*,
                                         double);
template int step_adjoint_coupled<double>(fs_grid*, const fs_state*, fs_state*, const double*, bool,
                                          fs_param_grad*, double);

}  // namespace fs
