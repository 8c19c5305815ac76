// Internal declarations of the fractional-step CUDA library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>

#include "fs.h"

#define FS_MAX_RADIX_STAGES 16

namespace fs {

// Boundary ghost rule for a tangential velocity component (§2.3.1, ghost values):
// Dirichlet sides (no-slip, inflow) reflect about the imposed value, the others copy.
__host__ __device__ inline bool bc_dirichlet(int kind) {
  return kind == FS_BC_NOSLIP || kind == FS_BC_INFLOW;
}

// Geometry handed to kernels by value.  x and z are uniform; y may be stretched.
template <typename T>
struct Geom {
  int dim, nx, ny, nz;
  int per[3];
  int bc[3][2];
  T bcv[3][2][3];
  T hx, hz, ihx, ihz;
  const T* ihy;   // 1 / h_y[j]           j in [0, ny)
  const T* ihfy;  // 1 / hf_y[j]          j in [0, ny]   (hf_y[ny] = hf_y[0] when periodic)
  const T* thy;   // theta_y[j]           j in [0, ny]
  const T* bforce;  // x-momentum source per y row, or nullptr
  T nu;
  __host__ __device__ int ext(int c, int d) const {
    int n = d == 0 ? nx : (d == 1 ? ny : nz);
    return n + ((c == d && !per[d]) ? 1 : 0);
  }
  __host__ __device__ int cells() const { return nx * ny * nz; }
};

// Load component c at integer position (i, j, k) that may lie one layer outside
// its storage in any direction: periodic directions wrap, tangential
// non-periodic directions apply the ghost rule, the component's own
// non-periodic direction clamps (that ghost is never used by an interior face).
template <typename T>
__device__ __forceinline__ T ldv(const Geom<T>& g, const T* __restrict__ u, int c, int i, int j, int k) {
  int idx[3] = {i, j, k};
  int e[3] = {g.ext(c, 0), g.ext(c, 1), g.ext(c, 2)};
  T sign = T(1), add = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int v = idx[d];
    if (v < 0 || v >= e[d]) {
      const int side = v < 0 ? 0 : 1;
      if (g.per[d]) {
        v = side ? v - e[d] : v + e[d];
      } else {
        v = side ? e[d] - 1 : 0;
        if (d != c && bc_dirichlet(g.bc[d][side])) {
          // ghost = 2 u_wall - (current value)
          add = T(2) * g.bcv[d][side][c] - add;
          sign = -sign;
        }
      }
      idx[d] = v;
    }
  }
  // A face on the component's own non-periodic boundary carries the imposed
  // normal velocity (0 on walls, U at the inflow) whatever the state holds;
  // only the outflow face is a state value.
  T raw;
  const int own = idx[c];
  if (!g.per[c] && (own == 0 || own == e[c] - 1) && g.bc[c][own == 0 ? 0 : 1] != FS_BC_OUTFLOW) {
    const int side = own == 0 ? 0 : 1;
    raw = g.bc[c][side] == FS_BC_INFLOW ? g.bcv[c][side][c] : T(0);
  } else {
    raw = u[idx[0] + (size_t)e[0] * (idx[1] + (size_t)e[1] * idx[2])];
  }
  return sign * raw + add;
}

// Rigid velocity V + omega x (r - r_c) at face position (px, py) (Eq. 23, solid points).
__device__ __forceinline__ void rigid_velocity(const double* body, double omega, double cx, double cy,
                                               double px, double py, double& vx, double& vy) {
  const double wx = body[0], wy = body[1];
  vx = body[2] - omega * (py - (cy + wy));
  vy = body[3] + omega * (px - (cx + wx));
}

// Inputs of the divergence D[(1 - eps) u* + eps u_c] of Eq. (9).
template <typename T>
struct DivArgs {
  Geom<T> g;
  const T* u[3];
  const uint8_t* flags[2];   // IB flags (2-D) or null
  const double* body;
  double omega, cx, cy;
  const double* xf;
  const double* yf;
  int vec4;                  // 1: periodic x, nx % 4 == 0, no IB: rows read four faces at a time
};

// Four consecutive values of a row whose start is 16-byte (float) / 32-byte (double) aligned.
template <typename T>
struct Vec4 {
  T v[4];
};
__device__ __forceinline__ Vec4<float> ld4(const float* __restrict__ p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Vec4<double> ld4(const double* __restrict__ p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, const Vec4<float>& a) {
  *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}
__device__ __forceinline__ void st4(double* p, const Vec4<double>& a) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a.v[0], a.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(a.v[2], a.v[3]);
}

// (1 - eps) u* + eps u_c on face t of component c: forced faces take the exact
// solid velocity u_c (Eq. 9), the others u*.
template <typename T>
__device__ __forceinline__ T blended(const DivArgs<T>& A, int c, int t, int i, int j) {
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
    return T(c == 0 ? vx : vy);
  }
  return A.u[c][t];
}

// Right-hand side of Eq. (9) at cell (i, j, k): sum_d (u_d[m+1] - u_d[m]) / h_d[m].
template <typename T>
__device__ __forceinline__ T div_at(const DivArgs<T>& A, int i, int j, int k) {
  const Geom<T>& g = A.g;
  T s;
  {
    const int ex = g.ext(0, 0);
    const int base = ex * (j + g.ny * k);
    const int ip = (i + 1 < ex) ? i + 1 : 0;
    s = (blended(A, 0, base + ip, ip, j) - blended(A, 0, base + i, i, j)) * g.ihx;
  }
  {
    const int ey = g.ext(1, 1);
    const int jp = (j + 1 < ey) ? j + 1 : 0;
    const int b0 = i + g.nx * ey * k;
    s += (blended(A, 1, b0 + g.nx * jp, i, jp) - blended(A, 1, b0 + g.nx * j, i, j)) * g.ihy[j];
  }
  if (g.dim == 3) {
    const int ez = g.ext(2, 2);
    const int kp = (k + 1 < ez) ? k + 1 : 0;
    const int b0 = i + g.nx * j;
    const int pl = g.nx * g.ny;
    s += (__ldg(A.u[2] + b0 + pl * kp) - __ldg(A.u[2] + b0 + pl * k)) * g.ihz;
  }
  return s;
}

// D u* at cells (i0 .. i0+3, j, k) for vec4 grids (periodic x, no IB).
template <typename T>
__device__ __forceinline__ Vec4<T> div4_at(const DivArgs<T>& A, int i0, int j, int k) {
  const Geom<T>& g = A.g;
  const int nx = g.nx;
  Vec4<T> s;
  {
    const T* row = A.u[0] + (size_t)nx * (j + g.ny * k);
    const Vec4<T> a = ld4(row + i0);
    const T e = __ldg(row + (i0 + 4 < nx ? i0 + 4 : 0));
    s.v[0] = (a.v[1] - a.v[0]) * g.ihx;
    s.v[1] = (a.v[2] - a.v[1]) * g.ihx;
    s.v[2] = (a.v[3] - a.v[2]) * g.ihx;
    s.v[3] = (e - a.v[3]) * g.ihx;
  }
  {
    const int ey = g.ext(1, 1);
    const int jp = (j + 1 < ey) ? j + 1 : 0;
    const T* pl = A.u[1] + (size_t)nx * ey * k + i0;
    const Vec4<T> a = ld4(pl + (size_t)nx * j), b = ld4(pl + (size_t)nx * jp);
    const T ih = g.ihy[j];
#pragma unroll
    for (int e = 0; e < 4; ++e) s.v[e] += (b.v[e] - a.v[e]) * ih;
  }
  if (g.dim == 3) {
    const int kp = (k + 1 < g.nz) ? k + 1 : 0;
    const size_t plane = (size_t)nx * g.ny;
    const T* col = A.u[2] + (size_t)nx * j + i0;
    const Vec4<T> a = ld4(col + plane * k), b = ld4(col + plane * kp);
#pragma unroll
    for (int e = 0; e < 4; ++e) s.v[e] += (b.v[e] - a.v[e]) * g.ihz;
  }
  return s;
}

// Workspace and plans owned by a grid (host side).
struct Plan1D {
  int n = 0;
  int nst = 0;
  int radix[FS_MAX_RADIX_STAGES];
  void* tw = nullptr;    // device twiddles exp(-2 pi i k / n), complex of the field precision
  void* dtw = nullptr;   // device DCT post-twiddles exp(-i pi k / (2 n)), field precision
};

struct IBDev {
  int nm = 0;
  int kernel = FS_ROMA3;
  double *X0 = nullptr, *Y0 = nullptr, *ds = nullptr;  // device, markers sorted by the cell of their rest position
  // edges of the rest contours, sorted by their lowest y (ey0), each from vertex a to vertex
  // next(a) in surface order: device arrays of ne = nm entries
  double *EAX = nullptr, *EAY = nullptr, *EBX = nullptr, *EBY = nullptr, *EY0 = nullptr;
  double ehmax = 0.0;                                  // largest edge height
  int* ebin = nullptr;                                 // first edge with ey0 >= ebin0 + k ebinh (nebin + 1)
  double ebin0 = 0.0, ebinh = 1.0;
  int nebin = 0;
  int* order = nullptr;                                // device, sorted position -> caller index
  // rest-frame cell bins of the sorted markers: bin_start[(cj - by0) * nbx + (ci - bx0)] is the
  // first sorted marker of cell (ci, cj); nbx * nby + 1 entries
  int* bin_start = nullptr;
  // sorted markers in grid units: rest cell (gi) and fraction in it (gf, field precision, x and y),
  // rest position minus the rotation centre (rel, field precision), and per (marker, component) the
  // interpolation weight factor dV_i / (F_N_i h_x h_y) of the step (wfac, field precision)
  int2* gi = nullptr;
  void* gf = nullptr;
  void* rel = nullptr;
  void* wfac = nullptr;
  void* dsh = nullptr;                                 // dV_i = ds_i h_x per sorted marker, field precision
  int bx0 = 0, by0 = 0, nbx = 0, nby = 0;
  unsigned* iblist = nullptr;                          // IB faces of the current step: (index << 1) | component
  unsigned* ibcount = nullptr;                         // their number (device)
  std::vector<int> horder;
  double centre[2] = {0, 0};
  double omega = 0;
  double mass = 0, k = 0, c = 0;
  int active[2] = {0, 0};
  uint8_t* flags[2] = {nullptr, nullptr};  // per face: bit0 solid, bit1 IB
  void* num[2] = {nullptr, nullptr};       // IB interpolation accumulators (field precision)
  void* den[2] = {nullptr, nullptr};
  void* f[2] = {nullptr, nullptr};         // direct-forcing term f of Eq. (5) (field precision)
  double* fn = nullptr;                    // F_N per marker and component (2 * nm)
  double* q = nullptr;                     // marker forces (2 * nm)
  double* part = nullptr;                  // per-block sums of the force kernel (3 per block)
  double* F = nullptr;                     // [Fx, Fy, torque]
  unsigned* ticket = nullptr;              // blocks finished in the force kernel (reset by its last block)
  bool have_forces = false;
  double poly_bb[4] = {0, 0, 0, 0};        // rest polygon bounding box xmin, xmax, ymin, ymax
};

// Static 3-D body made of axis-aligned boxes (ib3.cu): forced faces take zero velocity.
struct IB3Dev {
  int nbox = 0, nm = 0;
  int kernel = FS_ROMA3;
  double* boxes = nullptr;                  // device, nbox x 6
  double* X = nullptr;                      // device, marker x, y, z (SoA, 3 * nm)
  double* dV = nullptr;                     // device, marker volumes
  uint8_t* flags[3] = {nullptr, nullptr, nullptr};   // per face: bit0 solid, bit1 IB
  void* f[3] = {nullptr, nullptr, nullptr}; // direct-forcing term f of Eq. (5) (field precision)
  double* q = nullptr;                      // marker forces (3 * nm, SoA)
  double* F = nullptr;                      // [Fx, Fy, Fz]
  int* gi = nullptr;                        // marker cell index per direction (3 * nm, SoA)
  void* gf = nullptr;                       // fraction in the cell, field precision (3 * nm, SoA)
  double* part = nullptr;                   // per-block sums of the force gather
  unsigned* ticket = nullptr;               // blocks of the force gather finished
  bool have_forces = false;
};

}  // namespace fs

struct fs_grid {
  int dim = 2, nx = 1, ny = 1, nz = 1;
  int per[3] = {1, 1, 1};
  int bc[3][2];
  double bcv[3][2][3];
  double nu = 0, rho = 1;
  int conv = FS_CENTRAL2, scheme = FS_FE, prec = FS_FP64;
  double hx = 1, hz = 1;
  std::vector<double> xf[3], h[3], hf[3], th[3];
  std::vector<double> bforce;
  cudaStream_t stream = nullptr;
  // second stream and fork / join events of the split periodic-z Poisson solve (two halves of the
  // x spectrum as independent z / y / z chains)
  cudaStream_t ystream2 = nullptr;
  cudaEvent_t yev[2] = {nullptr, nullptr};
  int tune_ysplit = 0;
  long long launches = 0;

  // device metrics (both precisions)
  double *ihy64 = nullptr, *ihfy64 = nullptr, *thy64 = nullptr, *bf64 = nullptr;
  float *ihy32 = nullptr, *ihfy32 = nullptr, *thy32 = nullptr, *bf32 = nullptr;
  double *xf64[3] = {nullptr, nullptr, nullptr};   // face coordinates (IB positions)
  double *hy64 = nullptr;                          // cell widths in y (FP64)
  double *hfy64 = nullptr;                         // face spacings in y (FP64, ny + 1)

  // workspace (field precision)
  void* ustar[3] = {nullptr, nullptr, nullptr};
  void* ustage[3] = {nullptr, nullptr, nullptr};
  void* spec = nullptr;        // real-packed spectral / pressure work array (cells)
  double* scal = nullptr;      // small device scalars (flux sums, reductions)
  double* red = nullptr;       // reduction partials
  unsigned* dstatus = nullptr; // device status bits, set by kernels (1: a staged copy wait timed out)

  // Poisson plans
  fs::Plan1D px, py, pz;       // py: periodic y only
  int xmode = 0;               // 0: periodic DFT, 1: DCT-II
  int yspec = 0;               // 1: periodic (uniform) y, solved spectrally along y as well
  void* lamy = nullptr;        // field type: y eigenvalues -(2 - 2 cos(2 pi k / ny)) / hy^2 (ny)
  void* lamxz = nullptr;       // field type: x + z eigenvalue of each [lz][mx] index
  int nmx = 0, nlz = 1;        // eigenvalue table extents
  int cyclic = 0;
  double* ya = nullptr;        // a_j couplings (ny)
  double *tE = nullptr, *tCP = nullptr;   // [ny][nlz][nmx] segment factors e_j, c'_j
  double *tZV = nullptr, *tWV = nullptr;  // [ny][nlz][nmx] right / left spikes of each segment
  double *tMI = nullptr;                  // [4 ynseg^2][nlz][nmx] inverse of the 2 ynseg interface system
  int ynseg = 4;                          // segments per column of the partitioned y solve (4, 8 or 16)
  int ynarrow = 0;                        // 1: 8-column blocks; tE, tCP, tZV, tWV are then [nlam][ypitch]
  int ypitch = 0;                         // row count of the eigenvalue-major tables (ny rounded up to even)
  double hysum = 0.0;                     // sum of the y cell widths (zero-mode mean of the y solve)
  int yuniform = 0;                       // the y cells are all of one width
  // the twisted y solve shifts the zero mode's column to zero hy-weighted mean (the pressure's
  // gauge); off in the Poisson solves whose pressure is not written out, where only its gradient
  // is used and the column keeps the gauge of its factorisation (x = 0 at row 0)
  bool ygauge = true;
  int tune_ynseg = 0;                     // requested segment count (0: chosen from the grid's shape)
  bool tune_staged = true;                // shared-memory staged predictor where it applies
  int tune_pred_chunk = 0;                // staged predictor runs: 0 by grid size, -1 equal shares, > 0 aligned runs
  // twisted y solve (grids with many columns): two threads per column, tables per eigenvalue
  int ytwist = 0;                         // 1: the twisted solve runs instead of the partitioned one
  int tune_ytwist = -1;                   // -1: chosen from the grid's shape, 0: off, 1: on where it fits
  int ytw_cols = 64;                      // columns per block (64 or 32)
  int tune_ytw_cols = 0;                  // requested columns per block (0: chosen from ny)
  alignas(64) unsigned char ytw_map[128] = {};   // tensor map of the FP32 spectrum (CUtensorMap bytes)
  const void* ytw_map_ptr = nullptr;      // array and block width the map was encoded for
  int ytw_map_w = 0;
  bool ytw_map_ok = false;
  bool tune_ytile = true;                 // twisted solve: tensor-map tile loads where they apply
  int tune_xzplane = 1;                   // FP32 nx = nz of 64 or 128: x and z transforms fused per y position (1: one block, 2: a two-block cluster)
  int ytw_L = 0, ytw_R = 0;               // chain rows 0..L-1, positions per thread R = ceil(L / 2)
  int ytw_nlp = 0;                        // row pitch (eigenvalues) of the position-major tables
  double *twM = nullptr, *twE = nullptr, *twC = nullptr;   // [2 R + 4 kTwChunk][nlp], position-major
  double *twP = nullptr;                  // [nlz * nmx][4]
  double *twZ = nullptr;                  // [2 R + 4 kTwChunk][nlp] (periodic y)
  int* twK = nullptr;                     // [nlam] positions per thread where z matters (periodic y)
  double *twS = nullptr;                  // [nlz * nmx][4] (periodic y)
  // FP32 fields: the outward pass carries y = x / sigma (one multiply-add per row), sigma applied
  // in FP32 as the solution is narrowed
  float* twSig = nullptr;                 // [2 R + 4 kTwChunk][nlp] sigma per position, position-major
  double* twSig0 = nullptr;               // [2 R] sigma of the zero mode's column, FP64

  fs::IBDev ib;
  bool has_body = false;
  fs::IB3Dev ib3;
  bool has_ib3 = false;
  void* adj = nullptr;         // adjoint work buffers (adjoint.cu), allocated on first use
  void* cg = nullptr;          // conjugate-gradient workspace (cg.cu), allocated on first use
  // strong FSI coupling (fs_set_coupling): sub-iterations per step, tolerance, workspace
  int fsi_iters = 1;
  double fsi_tol = 1e-5;
  void* fsi_u[3] = {nullptr, nullptr, nullptr};   // velocity at time level n
  double* fsi_b = nullptr;     // [0..3] body at level n, [4..7] new iterate, [8] xi
  int fsi_last_iters = 0;
  double fsi_last_xi = 0.0;

  // launch parameters (fs_set_tuning; 0 = built-in default)
  int tune_stencil_bx = 0;     // x threads of the 2-D stencil blocks (32, 64, 128); blocks hold 256 threads
  int tune_fft_lines = 0;      // complex lines per FFT block (1..16)
  bool use_pdl = true;         // programmatic dependent launch of the step kernels
  int tune_pred_vw = 0;        // cells per thread of the FP32 predictor (1, 2 or 4; 0 = 4)
  int tune_zmarch = 0;         // planes per thread of the z-marching FP32 predictor (0: 8, 1: no march)
  // Smagorinsky LES (fs_set_les): constant, nu_t at centres and xy / xz / yz edges (field precision)
  double les_cs = 0.0;
  void* les_nu[4] = {nullptr, nullptr, nullptr, nullptr};

  // optional per-kernel timing (fs_profile_begin / fs_profile_end)
  bool prof_on = false;
  std::string prof_filter;
  std::vector<cudaEvent_t> prof_pool;
  size_t prof_used = 0;
  std::vector<std::string> prof_names;

  template <typename T> fs::Geom<T> geom() const;
};

namespace fs {
// kernels launchers (stencil.cu)
template <typename T> void launch_predictor(fs_grid* g, T* const* uin, T* const* un, T* const* out,
                                            double dt, double a, double b, const double* body_state);
template <typename T> void launch_outflow_flux(fs_grid* g, T* const* uin);
template <typename T> void launch_divergence(fs_grid* g, T* const* u, T* out, const double* body_state);
template <typename T> fs::DivArgs<T> make_div_args(fs_grid* g, T* const* u, const double* body_state);
template <typename T> void launch_correct(fs_grid* g, T* const* ustar, const T* phi, T* const* unew);
template <typename T> void launch_to_pressure(fs_grid* g, const T* phi, double* p, double scale);
template <typename T> void launch_diagnostics(fs_grid* g, T* const* u, double* out3);
// poisson.cu
template <typename T> void poisson_solve_inplace(fs_grid* g, T* data);
// Solve with the right-hand side D[(1 - eps) u* + eps u_c] formed inside the x transform (out: phi).
template <typename T> void poisson_solve_from_velocity(fs_grid* g, const fs::DivArgs<T>& div, T* data);
// ib.cu
template <typename T> void ib_prepare(fs_grid* g, const double* body_state);
// Marker forces, F and torque (Eq. 20); with `advance`, also the body ODE step
// (Eq. 12) of that state with the new force.
template <typename T> void ib_forces(fs_grid* g, double* body_state, double* advance = nullptr, double dt = 0.0);
void body_rk4(fs_grid* g, double* body_state, double dt);
// ib3.cu
template <typename T> void ib3_forces(fs_grid* g);
void free_ib3(fs_grid* g);
// adjoint.cu
// rv1, rv2: the RK3 stage states recorded by the forward step (then nothing is recomputed), or null
// dJdF_on_device: dJdF is a device pointer (else host)
template <typename T> int step_adjoint(fs_grid* g, const fs_state* st, fs_state* lam, const double* dJdF,
                                       fs_param_grad* pg, double dt, void* const* rv1 = nullptr,
                                       void* const* rv2 = nullptr, bool dJdF_on_device = false);
// adjoint of the strongly coupled (sub-iterated) FSI step by implicit differentiation
template <typename T> int step_adjoint_coupled(fs_grid* g, const fs_state* st, fs_state* lam, const double* dJdF,
                                               bool dJdF_on_device, fs_param_grad* pg, double dt);
// fs_api.cu: the strongly coupled forward-Euler FSI step (Algorithm 1)
template <typename T> int step_coupled(fs_grid* g, fs_state* st, double dt, bool want_p);
void free_adj_buffers(void* p);
// poisson.cu
size_t ysolve_smem(int ny, int nseg, int yc);
// rows per chunk of the twisted y solve; its tables carry 2 chunks of zero padding on each side
constexpr int kTwChunk = 16;
// errors
int set_error(int code, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);
}  // namespace fs

#define FS_LAUNCHED(g) ((g)->launches++)

// Block shape of the stencil kernels: bx threads along x, 256 / bx along y.
inline dim3 stencil_block(const fs_grid* G) {
  const int bx = G->tune_stencil_bx > 0 ? G->tune_stencil_bx : 32;
  return dim3(bx, 256 / bx);
}
inline dim3 stencil_grid(const fs_grid* G, int X, int Y) {
  const dim3 b = stencil_block(G);
  return dim3((X + b.x - 1) / b.x, (Y + b.y - 1) / b.y, G->nz);
}

namespace fs {
// Brackets one kernel launch with CUDA events on the grid's stream when
// profiling is on and the kernel name contains the profile filter.
struct ProfMark {
  fs_grid* g;
  int slot = -1;
  ProfMark(fs_grid* G, const char* name);
  ~ProfMark();
};
}  // namespace fs

namespace fs {
// Programmatic dependent launch: a kernel launched by launch_pdl may start
// while its predecessor on the stream drains; it must call pdl_wait() before
// its first access to global memory (a no-op for ordinary launches).
// pdl_trigger() lets the successor launch before this grid ends.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
void launch_pdl(fs_grid* G, const char* name, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                Args&&... args) {
  ProfMark pm(G, name);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = G->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = G->use_pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  G->launches++;
}
}  // namespace fs

// Launch with accounting: FS_LAUNCH(grid, "name", kernel<<<...>>>(...));
#define FS_LAUNCH(G, NAME, ...)        \
  do {                                 \
    fs::ProfMark fs_pm_((G), (NAME));  \
    __VA_ARGS__;                       \
    FS_LAUNCHED(G);                    \
  } while (0)
