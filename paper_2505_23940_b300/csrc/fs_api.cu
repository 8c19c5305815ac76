// C ABI of the fractional-step library (include/fs.h): grid set-up (metrics,
// transform plans, tridiagonal factor tables), workspaces and the order of
// kernels in one time step (Eqs. 4-10 and 18-23, 12 of the paper).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fs_internal.cuh"

namespace fs {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FS_OK;
  return set_error(FS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

ProfMark::ProfMark(fs_grid* G, const char* name) : g(G) {
  if (!G->prof_on) return;
  if (!G->prof_filter.empty() && std::string(name).find(G->prof_filter) == std::string::npos) return;
  if (G->prof_used + 2 > G->prof_pool.size()) {
    for (int q = 0; q < 64; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      G->prof_pool.push_back(e);
    }
  }
  slot = (int)G->prof_used;
  G->prof_used += 2;
  G->prof_names.push_back(name);
  cudaEventRecord(G->prof_pool[slot], G->stream);
}

ProfMark::~ProfMark() {
  if (slot >= 0) cudaEventRecord(g->prof_pool[slot + 1], g->stream);
}

namespace {

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc((void**)p, (n > 0 ? n : 1) * sizeof(T));
}

template <typename T>
cudaError_t upload(T** p, const std::vector<T>& v) {
  cudaError_t e = dalloc(p, v.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T>
std::vector<T> cast(const std::vector<double>& v) {
  return std::vector<T>(v.begin(), v.end());
}

bool factorize(int n, Plan1D& p) {
  p.n = n;
  p.nst = 0;
  int m = n;
  while (m % 4 == 0 && m > 4) {
    if (p.nst >= FS_MAX_RADIX_STAGES) return false;
    p.radix[p.nst++] = 4;
    m /= 4;
  }
  const int primes[] = {4, 2, 3, 5, 7, 11, 13};
  for (int q : primes) {
    while (m % q == 0) {
      if (p.nst >= FS_MAX_RADIX_STAGES) return false;
      p.radix[p.nst++] = q;
      m /= q;
    }
  }
  return m == 1;
}

template <typename T>
cudaError_t make_twiddles(Plan1D& p) {
  const int n = p.n;
  std::vector<T> tw(2 * n), dtw(2 * n);
  for (int k = 0; k < n; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)n;
    tw[2 * k] = (T)std::cos(a);
    tw[2 * k + 1] = (T)(-std::sin(a));
    const double b = M_PI * (double)k / (2.0 * (double)n);
    dtw[2 * k] = (T)std::cos(b);
    dtw[2 * k + 1] = (T)(-std::sin(b));
  }
  cudaError_t e = upload((T**)&p.tw, tw);
  if (e != cudaSuccess) return e;
  return upload((T**)&p.dtw, dtw);
}

bool uniform(const std::vector<double>& h) {
  for (double v : h)
    if (std::fabs(v - h[0]) > 1e-12 * std::fabs(h[0])) return false;
  return true;
}

size_t comp_size(const fs_grid* G, int c) {
  size_t s = 1;
  const int n[3] = {G->nx, G->ny, G->nz};
  for (int d = 0; d < 3; ++d) s *= (size_t)(n[d] + ((c == d && !G->per[d]) ? 1 : 0));
  return s;
}

size_t elem_size(const fs_grid* G) { return G->prec == FS_MIXED ? sizeof(float) : sizeof(double); }

// FP64 tables of the twisted y solve (poisson.cu: ytwist_kernel), per eigenvalue
// index li = lz * nmx + mx, from the couplings a_j (row j to j - 1) and c_j (row j
// to j + 1; both wrap around on periodic y) and the diagonal b_j = lambda - a_j - c_j.
// Chain rows 0..L-1 (L = ny, or ny - 1 on periodic y where row ny - 1 is bordered
// off); the upper elimination runs over rows 0..k, the lower over L-1..k+1:
//   upper: beta_j = b_j - a_j c_{j-1} / beta_{j-1},  M_j = -a_j / beta_{j-1}   (j = 1..k)
//          E_j = 1 / beta_j,  C_j = -c_j / beta_j                            (j = 0..k-1)
//   lower: beta'_j = b_j - c_j a_{j+1} / beta'_{j+1},  M_j = -c_j / beta'_{j+1} (j = L-2..k+1)
//          E_j = 1 / beta'_j,  C_j = -a_j / beta'_j                          (j = k+2..L-1)
//   P = inverse of [[beta_k, c_k], [a_{k+1}, beta'_{k+1}]]
// The singular zero mode pins x_0 = 0: 1 / beta_0 taken as 0, no coupling into row 0
// (the corner couplings of row 0 and row ny - 1 vanish).
// Periodic y also stores z = A''^-1 u (u_0 = a_0, u_{L-1} = c_{L-1}: the coupling
// column of x_{ny-1}), computed with the same tables, and S = (c_{ny-1}, a_{ny-1},
// 1 / (b_{ny-1} - c_{ny-1} z_0 - a_{ny-1} z_{ny-2})).
// Layout: M, E, C, Z position-major [rows][nlp]: each thread of a column owns R = ceil(L / 2)
// positions, the upper rows 0..R-1 (k = R - 1), the lower from position R: when L is odd first
// an inert slot (M = 0, E = 1, C = 0, z = 0; it carries the bordered row ny - 1 on periodic y),
// then rows L-1 down to R.  The rows are 2 kTwChunk zero rows, the 2 R positions, 2 kTwChunk
// zero rows; nlp >= nlam + 72 leaves room for the kernel's L2 prefetch of a block's segment.
// P and S are [nlam][4].
// FP32 fields (mixed precision) take the outward pass in scaled form: with sigma_p = E_p (1 at
// each thread's last position, whose x the 2x2 system gives, and at the inert slot; 0 at the
// zero mode's pinned row) and y_p = x_p / sigma_p, the substitution x_p = E_p g_p + C_p x_{p+1}
// becomes y_p = g_p + C'_p y_{p+1}, C'_p = C_p s_{p+1} / s_p (s = sigma, 1 where sigma = 0):
// one multiply-add per row instead of a multiply and a multiply-add.  The cyclic correction
// x = sigma (y - xi z / sigma) then uses z / sigma, and S0, S1 absorb sigma at rows 0 and L - 1.
// sigma is tabulated in FP32 and applied in FP32 to the narrowed solution (the zero mode's
// column in FP64, for its mean); E is not stored for such grids.
int build_twisted_tables(fs_grid* G, const std::vector<double>& a, const std::vector<double>& c) {
  const int nx = G->nx, ny = G->ny, nz = G->nz;
  const int nlam = G->nmx * G->nlz;
  const bool cyc = G->cyclic != 0;
  const int L = cyc ? ny - 1 : ny, R = (L + 1) / 2, k = R - 1;
  const bool odd = (L & 1) != 0;
  const int front = 2 * kTwChunk;
  const int rows = 2 * R + 4 * kTwChunk;
  const int nlp = (nlam + 72 + 1) & ~1;
  G->ytw_L = L;
  G->ytw_R = R;
  G->ytw_nlp = nlp;
  auto at = [&](int p, int li) { return (size_t)(front + p) * nlp + li; };
  auto pos = [&](int j) { return j < R ? j : R + (odd ? 1 : 0) + (L - 1 - j); };
  std::vector<double> M((size_t)rows * nlp, 0.0), E((size_t)rows * nlp, 0.0), C((size_t)rows * nlp, 0.0);
  std::vector<double> P((size_t)4 * nlam, 0.0), Z, S;
  std::vector<int> K(nlam, 0);
  if (cyc) {
    Z.assign((size_t)rows * nlp, 0.0);
    S.assign((size_t)4 * nlam, 0.0);
  }
  const bool yform = G->prec == FS_MIXED;
  std::vector<float> SG;
  std::vector<double> SG0, sc(2 * R), sig(2 * R);
  if (yform) {
    SG.assign((size_t)rows * nlp, 0.0f);
    SG0.assign(2 * R, 0.0);
  }
  std::vector<double> aa(ny), cc(ny), bb(ny), beta(ny), e(ny), rhs(ny), x(ny), gh(ny);
  std::vector<double> m(ny), ee(ny), cm(ny);
  for (int mx = 0; mx < G->nmx; ++mx) {
    const double lx = G->xmode == 1 ? -(2.0 - 2.0 * std::cos(M_PI * mx / nx)) / (G->hx * G->hx)
                                    : -(2.0 - 2.0 * std::cos(2.0 * M_PI * mx / nx)) / (G->hx * G->hx);
    for (int lz = 0; lz < G->nlz; ++lz) {
      const double lzv = G->dim == 3 ? -(2.0 - 2.0 * std::cos(2.0 * M_PI * lz / nz)) / (G->hz * G->hz) : 0.0;
      const double lam = lx + lzv;
      const int li = lz * G->nmx + mx;
      const bool sing = (mx == 0 && lz == 0);
      for (int j = 0; j < ny; ++j) {
        aa[j] = a[j];
        cc[j] = c[j];
        bb[j] = -(a[j] + c[j]) + lam;
      }
      if (sing) {
        aa[0] = 0.0;
        cc[0] = 0.0;
        if (cyc) cc[ny - 1] = 0.0;
      }
      // upper elimination
      e[0] = sing ? 0.0 : 1.0 / bb[0];
      beta[0] = bb[0];
      m[0] = 0.0;
      for (int j = 1; j <= k; ++j) {
        beta[j] = bb[j] - aa[j] * cc[j - 1] * e[j - 1];
        e[j] = 1.0 / beta[j];
        m[j] = -aa[j] * e[j - 1];
      }
      for (int j = 0; j < k; ++j) {
        ee[j] = e[j];
        cm[j] = -cc[j] * e[j];
      }
      // lower elimination
      beta[L - 1] = bb[L - 1];
      e[L - 1] = 1.0 / beta[L - 1];
      m[L - 1] = 0.0;
      for (int j = L - 2; j > k; --j) {
        beta[j] = bb[j] - cc[j] * aa[j + 1] * e[j + 1];
        e[j] = 1.0 / beta[j];
        m[j] = -cc[j] * e[j + 1];
      }
      for (int j = k + 2; j < L; ++j) {
        ee[j] = e[j];
        cm[j] = -aa[j] * e[j];
      }
      ee[k] = ee[k + 1] = cm[k] = cm[k + 1] = 0.0;
      const double det = beta[k] * beta[k + 1] - cc[k] * aa[k + 1];
      const double p[4] = {beta[k + 1] / det, -cc[k] / det, -aa[k + 1] / det, beta[k] / det};
      for (int q = 0; q < 4; ++q) P[(size_t)li * 4 + q] = p[q];
      for (int j = 0; j < L; ++j) {
        const size_t o = at(pos(j), li);
        M[o] = m[j];
        E[o] = ee[j];
        C[o] = cm[j];
      }
      if (odd) E[at(R, li)] = 1.0;   // the inert slot keeps its value
      if (cyc) {
        // z = A''^-1 u by the same two-sided sweeps
        for (int j = 0; j < L; ++j) rhs[j] = 0.0;
        rhs[0] += aa[0];
        rhs[L - 1] += cc[L - 1];
        gh[0] = rhs[0];
        for (int j = 1; j <= k; ++j) gh[j] = rhs[j] + m[j] * gh[j - 1];
        gh[L - 1] = rhs[L - 1];
        for (int j = L - 2; j > k; --j) gh[j] = rhs[j] + m[j] * gh[j + 1];
        x[k] = p[0] * gh[k] + p[1] * gh[k + 1];
        x[k + 1] = p[2] * gh[k] + p[3] * gh[k + 1];
        for (int j = k - 1; j >= 0; --j) x[j] = ee[j] * gh[j] + cm[j] * x[j + 1];
        for (int j = k + 2; j < L; ++j) x[j] = ee[j] * gh[j] + cm[j] * x[j - 1];
        for (int j = 0; j < L; ++j) Z[at(pos(j), li)] = x[j];
        // positions (from each thread's first) beyond which |z| < 2^-56 max |z|: the correction
        // x = y - xi z changes nothing there at FP64 precision and is skipped
        double zmax = 0.0;
        for (int j = 0; j < L; ++j) zmax = std::max(zmax, std::fabs(x[j]));
        int kz = 1;
        for (int p = 0; p < 2 * R; ++p) {
          const int j = p < R ? p : (odd && p == R ? -1 : L - 1 - (p - R - (odd ? 1 : 0)));
          if (j >= 0 && std::fabs(x[j]) > std::ldexp(zmax, -56)) kz = std::max(kz, (p < R ? p : p - R) + 1);
        }
        K[li] = kz;
        const double sigma = bb[ny - 1] - cc[ny - 1] * x[0] - aa[ny - 1] * x[L - 1];
        S[(size_t)li * 4 + 0] = cc[ny - 1];
        S[(size_t)li * 4 + 1] = aa[ny - 1];
        S[(size_t)li * 4 + 2] = 1.0 / sigma;
      }
      if (yform) {
        for (int p = 0; p < 2 * R; ++p) {
          const double ev = E[at(p, li)];
          const bool last = p == R - 1 || p == 2 * R - 1;
          sig[p] = last ? 1.0 : ev;
          sc[p] = sig[p] != 0.0 ? sig[p] : 1.0;
        }
        // the outward pass of each thread: local positions R - 2 .. 0, each coupled to the next
        for (int half = 0; half < 2; ++half)
          for (int i = 0; i + 1 < R; ++i) {
            const int p = half * R + i;
            C[at(p, li)] = C[at(p, li)] * sc[p + 1] / sc[p];
          }
        for (int p = 0; p < 2 * R; ++p) {
          SG[at(p, li)] = (float)sig[p];
          E[at(p, li)] = 0.0;
          if (cyc) Z[at(p, li)] = sig[p] != 0.0 ? Z[at(p, li)] / sig[p] : 0.0;
        }
        if (cyc) {
          S[(size_t)li * 4 + 0] *= sig[pos(0)];
          S[(size_t)li * 4 + 1] *= sig[pos(L - 1)];
        }
        if (li == 0) SG0 = sig;
      }
    }
  }
  if (yform && (upload(&G->twSig, SG) != cudaSuccess || upload(&G->twSig0, SG0) != cudaSuccess))
    return set_error(FS_ERR_CUDA, "allocating tridiagonal tables");
  if (upload(&G->twM, M) != cudaSuccess || (!yform && upload(&G->twE, E) != cudaSuccess) ||
      upload(&G->twC, C) != cudaSuccess ||
      upload(&G->twP, P) != cudaSuccess ||
      (cyc && (upload(&G->twZ, Z) != cudaSuccess || upload(&G->twS, S) != cudaSuccess ||
               upload(&G->twK, K) != cudaSuccess)))
    return set_error(FS_ERR_CUDA, "allocating tridiagonal tables");
  return FS_OK;
}

// FP64 tables of the partitioned y solve, one column per eigenvalue index:
// for each of the NSEG segments of every column, the local Thomas factors of the
// segment's block (e_j = 1 / beta_j, c'_j) and its right / left spikes v, w
// (the block's response to its coupling with the next / previous segment).
// The singular zero mode replaces row 0 by phi_0 = 0 (e_0 = 0, no couplings).
// NSEG is 4, or 8 for ny >= 192 and for grids with fewer 32-column blocks than
// two per SM (2-D grids): shorter sequential sweeps (16 segments cost more in
// the denser interface solve than they save).
int build_tables(fs_grid* G) {
  const int nx = G->nx, ny = G->ny, nz = G->nz;
  G->ytwist = 0;
  if (G->tune_ynseg > 0) {
    G->ynseg = G->tune_ynseg;
  } else {
    const long blocks = (long)((nx + 31) / 32) * (G->dim == 3 ? nz : 1);
    // sweeps of about 32 rows: 8 segments from ny = 192 on (256^3 channel: 296 against 382 us),
    // and on grids with too few columns for two blocks per SM (2-D: latency-bound)
    G->ynseg = ((blocks < 2 * 148 && ny >= 8 * 8) || ny >= 192) ? 8 : 4;
  }
  const int NSEG = G->ynseg;
  G->nmx = G->xmode == 1 ? nx : nx / 2 + 1;
  G->nlz = G->dim == 3 ? nz / 2 + 1 : 1;
  const int nlam = G->nmx * G->nlz;
  if (G->yspec) {
    // periodic y is uniform: the y operator is circulant and diagonal in the DFT basis
    const double hy = G->h[1][0];
    std::vector<double> ly(ny), lxz(nlam);
    for (int k = 0; k < ny; ++k) ly[k] = -(2.0 - 2.0 * std::cos(2.0 * M_PI * k / ny)) / (hy * hy);
    for (int mx = 0; mx < G->nmx; ++mx)
      for (int lz = 0; lz < G->nlz; ++lz) {
        const double lx = G->xmode == 1 ? -(2.0 - 2.0 * std::cos(M_PI * mx / nx)) / (G->hx * G->hx)
                                        : -(2.0 - 2.0 * std::cos(2.0 * M_PI * mx / nx)) / (G->hx * G->hx);
        const double lzv = G->dim == 3 ? -(2.0 - 2.0 * std::cos(2.0 * M_PI * lz / nz)) / (G->hz * G->hz) : 0.0;
        lxz[lz * G->nmx + mx] = lx + lzv;
      }
    const bool ok = G->prec == FS_MIXED
                        ? (upload((float**)&G->lamy, cast<float>(ly)) == cudaSuccess &&
                           upload((float**)&G->lamxz, cast<float>(lxz)) == cudaSuccess)
                        : (upload((double**)&G->lamy, ly) == cudaSuccess &&
                           upload((double**)&G->lamxz, lxz) == cudaSuccess);
    return ok ? FS_OK : set_error(FS_ERR_CUDA, "allocating eigenvalue tables");
  }
  const std::vector<double>& h = G->h[1];
  const std::vector<double>& hf = G->hf[1];
  G->hysum = 0.0;
  for (int j = 0; j < ny; ++j) G->hysum += h[j];
  G->yuniform = uniform(h) ? 1 : 0;
  std::vector<double> a(ny), c(ny);
  for (int j = 0; j < ny; ++j) {
    a[j] = 1.0 / (hf[j] * h[j]);        // coupling of row j to j - 1 (row 0: wraps to ny - 1)
    c[j] = 1.0 / (hf[j + 1] * h[j]);    // coupling of row j to j + 1 (row ny - 1: wraps to 0)
  }
  if (!G->per[1]) {
    a[0] = 0.0;           // G p . n = 0 on the walls
    c[ny - 1] = 0.0;
  }
  G->cyclic = G->per[1];
  {
    const long columns = (long)nx * (G->dim == 3 ? nz : 1);
    const int L = G->cyclic ? ny - 1 : ny;
    // by default where a 64-column block fits an SM (ny <= 292) on a grid that fills every SM.
    // Measured per mixed step: isotropic 128^3 (periodic y) 0.237-0.242 against 0.286 ms, the
    // wall-bounded 192 x 129 x 128 channel 0.161-0.165 against 0.173 ms, 256^3 (periodic y)
    // 1.88 against 1.91 ms.
    const bool want = G->tune_ytwist < 0 ? (columns >= 148L * 64 && ny <= 292) : G->tune_ytwist == 1;
    // shared memory holds the block's columns (ny + 1 positions) in FP64 plus their FP32 copy:
    // 64 columns (two blocks per SM while ny <= 148, one up to ny = 292), else 32 (ny <= 585).
    // A block's warp 0 .. 3 run on the SM's four sub-partitions and its first W / 16 warps
    // sweep: 64 columns keep an FP64 pipe busy on every sub-partition (256^3 periodic, FP64 y:
    // 1.88 ms per step with one 64-column block per SM, 1.92 with two 32-column blocks, 1.91
    // partitioned)
    G->ytw_cols = (size_t)(ny + 1) * 64 * 12 <= 220 * 1024 ? 64 : 32;
    if (G->tune_ytw_cols > 0) G->ytw_cols = G->tune_ytw_cols;
    // periodic y needs an odd chain (ny even): the lower thread's first slot holds the bordered row
    G->ytwist = L >= 4 && (size_t)(ny + 1) * G->ytw_cols * 12 <= 220 * 1024 && want && !(G->cyclic && (ny & 1));
    if (G->ytwist) return build_twisted_tables(G, a, c);
  }
  const int NRED = 2 * NSEG;
  std::vector<double> E((size_t)ny * nlam), CP((size_t)ny * nlam), V((size_t)ny * nlam), W((size_t)ny * nlam);
  std::vector<double> MI((size_t)NRED * NRED * nlam);
  std::vector<double> aa(ny), cc(ny), dd(ny), e(ny), cp(ny), dp(ny), x(ny);
  std::vector<double> acoef(ny);
  for (int j = 0; j < ny; ++j) acoef[j] = a[j];
  for (int mx = 0; mx < G->nmx; ++mx) {
    const double lx = G->xmode == 1 ? -(2.0 - 2.0 * std::cos(M_PI * mx / nx)) / (G->hx * G->hx)
                                    : -(2.0 - 2.0 * std::cos(2.0 * M_PI * mx / nx)) / (G->hx * G->hx);
    for (int lz = 0; lz < G->nlz; ++lz) {
      const double lzv = G->dim == 3 ? -(2.0 - 2.0 * std::cos(2.0 * M_PI * lz / nz)) / (G->hz * G->hz) : 0.0;
      const double lam = lx + lzv;
      const int li = lz * G->nmx + mx;   // [j][lz][mx] layout
      const bool sing = (mx == 0 && lz == 0);
      for (int j = 0; j < ny; ++j) {
        aa[j] = a[j];
        cc[j] = c[j];
        dd[j] = -(a[j] + c[j]) + lam;
      }
      if (sing) {         // phi_0 = 0 replaces row 0; no coupling reaches row 0
        aa[0] = 0.0;
        cc[0] = 0.0;
        if (G->cyclic) cc[ny - 1] = 0.0;
      }
      for (int g = 0; g < NSEG; ++g) {
        const int r0 = (g * ny) / NSEG, r1 = ((g + 1) * ny) / NSEG;
        if (r1 <= r0) continue;
        for (int j = r0; j < r1; ++j) {
          const double beta = dd[j] - (j > r0 ? acoef[j] * cp[j - 1] : 0.0);
          e[j] = (sing && j == 0) ? 0.0 : 1.0 / beta;
          cp[j] = j < r1 - 1 ? cc[j] * e[j] : 0.0;
        }
        // spikes: A_g^-1 (a_{r0} e_first), A_g^-1 (c_{r1-1} e_last)
        for (int which = 0; which < 2; ++which) {
          for (int j = r0; j < r1; ++j) {
            const double rhs = which == 0 ? (j == r0 ? aa[r0] : 0.0) : (j == r1 - 1 ? cc[r1 - 1] : 0.0);
            dp[j] = j == r0 ? rhs * e[j] : (rhs - acoef[j] * dp[j - 1]) * e[j];
          }
          x[r1 - 1] = dp[r1 - 1];
          for (int j = r1 - 2; j >= r0; --j) x[j] = dp[j] - cp[j] * x[j + 1];
          for (int j = r0; j < r1; ++j) (which == 0 ? W : V)[(size_t)j * nlam + li] = x[j];
        }
        for (int j = r0; j < r1; ++j) {
          E[(size_t)j * nlam + li] = e[j];
          CP[(size_t)j * nlam + li] = cp[j];
        }
      }
      // interface system X_p + v X_{p+1} + w Y_{p-1} = y_first, Y_p + v X_{p+1} + w Y_{p-1} = y_last
      std::vector<std::vector<double>> M(NRED, std::vector<double>(2 * NRED));
      for (int r = 0; r < NRED; ++r)
        for (int q = 0; q < 2 * NRED; ++q) M[r][q] = (q == r || q == r + NRED) ? 1.0 : 0.0;
      for (int g = 0; g < NSEG; ++g) {
        const int r0 = (g * ny) / NSEG, r1 = ((g + 1) * ny) / NSEG;
        if (r1 <= r0) continue;
        const int gn = g + 1 < NSEG ? g + 1 : 0, gp = g > 0 ? g - 1 : NSEG - 1;
        const bool hn = g + 1 < NSEG || G->cyclic, hp = g > 0 || G->cyclic;
        const int rows[2] = {r0, r1 - 1};
        for (int hh = 0; hh < 2; ++hh) {
          const int row = 2 * g + hh;
          if (hn) M[row][2 * gn] += V[(size_t)rows[hh] * nlam + li];
          if (hp) M[row][2 * gp + 1] += W[(size_t)rows[hh] * nlam + li];
        }
      }
      // Gauss-Jordan with partial pivoting on [M | I]
      for (int k = 0; k < NRED; ++k) {
        int piv = k;
        for (int r = k + 1; r < NRED; ++r)
          if (std::fabs(M[r][k]) > std::fabs(M[piv][k])) piv = r;
        if (piv != k)
          for (int q = 0; q < 2 * NRED; ++q) std::swap(M[k][q], M[piv][q]);
        const double inv = 1.0 / M[k][k];
        for (int q = 0; q < 2 * NRED; ++q) M[k][q] *= inv;
        for (int r = 0; r < NRED; ++r) {
          if (r == k || M[r][k] == 0.0) continue;
          const double f = M[r][k];
          for (int q = 0; q < 2 * NRED; ++q) M[r][q] -= f * M[k][q];
        }
      }
      for (int r = 0; r < NRED; ++r)
        for (int q = 0; q < NRED; ++q) MI[(size_t)(r * NRED + q) * nlam + li] = M[r][NRED + q];
    }
  }
  // grids with too few 32-column blocks to fill the SMs solve in 8-column blocks that copy their
  // columns' tables into shared memory: those tables are stored eigenvalue-major, one contiguous
  // (padded) column per eigenvalue index
  const long blocks32 = (long)((nx + 31) / 32) * (G->dim == 3 ? nz : 1);
  G->ypitch = ny + (ny & 1);
  G->ynarrow = blocks32 < 148 && ysolve_smem(ny, NSEG, 8) <= 200 * 1024;
  if (G->ynarrow) {
    auto transpose = [&](const std::vector<double>& t) {
      std::vector<double> o((size_t)nlam * G->ypitch, 0.0);
      for (int j = 0; j < ny; ++j)
        for (int l = 0; l < nlam; ++l) o[(size_t)l * G->ypitch + j] = t[(size_t)j * nlam + l];
      return o;
    };
    E = transpose(E);
    CP = transpose(CP);
    V = transpose(V);
    W = transpose(W);
    acoef.resize(G->ypitch, 0.0);
  }
  if (upload(&G->ya, acoef) != cudaSuccess || upload(&G->tE, E) != cudaSuccess || upload(&G->tCP, CP) != cudaSuccess ||
      upload(&G->tZV, V) != cudaSuccess || upload(&G->tWV, W) != cudaSuccess || upload(&G->tMI, MI) != cudaSuccess)
    return set_error(FS_ERR_CUDA, "allocating tridiagonal tables");
  return FS_OK;
}

void free_ytables(fs_grid* G) {
  double** t[12] = {&G->ya, &G->tE, &G->tCP, &G->tZV, &G->tWV, &G->tMI,
                    &G->twM, &G->twE, &G->twC, &G->twP, &G->twZ, &G->twS};
  for (double** p : t) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  if (G->twK) cudaFree(G->twK);
  G->twK = nullptr;
  if (G->twSig) cudaFree(G->twSig);
  G->twSig = nullptr;
  if (G->twSig0) cudaFree(G->twSig0);
  G->twSig0 = nullptr;
}

void free_all(fs_grid* G) {
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  if (G->yev[0]) cudaEventDestroy(G->yev[0]);
  if (G->yev[1]) cudaEventDestroy(G->yev[1]);
  if (G->ystream2) cudaStreamDestroy(G->ystream2);
  G->yev[0] = G->yev[1] = nullptr;
  G->ystream2 = nullptr;
  F(G->ihy64); F(G->ihfy64); F(G->thy64); F(G->bf64);
  F(G->ihy32); F(G->ihfy32); F(G->thy32); F(G->bf32);
  for (int d = 0; d < 3; ++d) F(G->xf64[d]);
  F(G->hy64); F(G->hfy64);
  for (int c = 0; c < 3; ++c) { F(G->ustar[c]); F(G->ustage[c]); }
  F(G->spec); F(G->scal); F(G->red); F(G->cg); F(G->dstatus);
  for (int c = 0; c < 3; ++c) F(G->fsi_u[c]);
  F(G->fsi_b);
  for (int q = 0; q < 4; ++q) F(G->les_nu[q]);
  F(G->px.tw); F(G->px.dtw); F(G->py.tw); F(G->py.dtw); F(G->pz.tw); F(G->pz.dtw);
  F(G->lamy); F(G->lamxz);
  free_ytables(G);
  IBDev& B = G->ib;
  F(B.X0); F(B.Y0); F(B.ds); F(B.order);
  F(B.EAX); F(B.EAY); F(B.EBX); F(B.EBY); F(B.EY0); F(B.bin_start); F(B.iblist); F(B.ibcount); F(B.ebin);
  F(B.gi); F(B.gf); F(B.rel); F(B.wfac); F(B.dsh);
  for (int c = 0; c < 2; ++c) { F(B.flags[c]); F(B.num[c]); F(B.den[c]); F(B.f[c]); }
  F(B.fn); F(B.q); F(B.part); F(B.F); F(B.ticket);
}

void free_body(fs_grid* G) {
  IBDev& B = G->ib;
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  F(B.X0); F(B.Y0); F(B.ds); F(B.order);
  F(B.EAX); F(B.EAY); F(B.EBX); F(B.EBY); F(B.EY0); F(B.bin_start); F(B.iblist); F(B.ibcount); F(B.ebin);
  F(B.gi); F(B.gf); F(B.rel); F(B.wfac); F(B.dsh);
  for (int c = 0; c < 2; ++c) { F(B.flags[c]); F(B.num[c]); F(B.den[c]); F(B.f[c]); }
  F(B.fn); F(B.q); F(B.part); F(B.F); F(B.ticket);
  B = IBDev();
  G->has_body = false;
}

// rec1, rec2: where an RK3 step leaves its two stage states (null: the grid's stage buffer)
template <typename T>
void step_once(fs_grid* G, fs_state* st, double dt, bool want_p, void* const* rec1 = nullptr,
               void* const* rec2 = nullptr) {
  T* u[3] = {(T*)st->u[0], (T*)st->u[1], (T*)(G->dim == 3 ? st->u[2] : nullptr)};
  T* us[3] = {(T*)G->ustar[0], (T*)G->ustar[1], (T*)G->ustar[2]};
  T* spec = (T*)G->spec;
  if (G->scheme == FS_RK3) {
    T* v[3] = {(T*)G->ustage[0], (T*)G->ustage[1], (T*)G->ustage[2]};
    T* v1[3] = {v[0], v[1], v[2]};
    T* v2[3] = {v[0], v[1], v[2]};
    if (rec1 && rec2)
      for (int c = 0; c < G->dim; ++c) {
        v1[c] = (T*)rec1[c];
        v2[c] = (T*)rec2[c];
      }
    const double A[3] = {0.0, 0.75, 1.0 / 3.0}, Bc[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int s = 0; s < 3; ++s) {
      T* const* in = s == 0 ? u : (s == 1 ? v1 : v2);
      launch_predictor<T>(G, in, u, us, dt, A[s], Bc[s], nullptr);
      G->ygauge = want_p && s == 2;              // only the written-out pressure needs its gauge
      poisson_solve_from_velocity<T>(G, make_div_args<T>(G, us, nullptr), spec);
      G->ygauge = true;
      launch_correct<T>(G, us, spec, s == 2 ? u : (s == 0 ? v1 : v2));
    }
    if (want_p) launch_to_pressure<T>(G, spec, st->p, G->rho / (Bc[2] * dt));
    return;
  }
  if (G->has_body) ib_prepare<T>(G, st->body);
  launch_outflow_flux<T>(G, u);
  launch_predictor<T>(G, u, nullptr, us, dt, 0.0, 1.0, st->body);
  G->ygauge = want_p;
  poisson_solve_from_velocity<T>(G, make_div_args<T>(G, us, st->body), spec);
  G->ygauge = true;
  launch_correct<T>(G, us, spec, u);
  if (want_p) launch_to_pressure<T>(G, spec, st->p, G->rho / dt);
  if (G->has_body) {
    ib_forces<T>(G, st->body, st->body, dt);
  }
  if (G->has_ib3) ib3_forces<T>(G);
}

// xi = |w_new - w_it|^2 / |w_it|^2 (|w_new - w_it|^2 while w_it = 0); the iterate
// st := the new body state.
__global__ void couple_kernel(double* __restrict__ st, const double* __restrict__ nb, double* __restrict__ xi) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double num = 0.0, den = 0.0;
  for (int d = 0; d < 2; ++d) {
    const double dw = nb[d] - st[d];
    num += dw * dw;
    den += st[d] * st[d];
  }
  *xi = den > 0.0 ? num / den : num;
  for (int q = 0; q < 4; ++q) st[q] = nb[q];
}

}  // namespace

// Strongly coupled forward-Euler FSI step (§2.3.3, Algorithm 1): sub-iterate the
// fluid solve (kinematics of the current body iterate, from u^n) and the body
// ODE (from the body at level n, with the force of that solve) until the
// relative change of the displacement falls below fsi_tol, at most fsi_iters
// fluid solves.  The convergence test reads xi on the host once per
// sub-iteration.
template <typename T>
int step_coupled(fs_grid* G, fs_state* st, double dt, bool want_p) {
  const size_t es = sizeof(T);
  size_t n[3];
  for (int c = 0; c < G->dim; ++c) n[c] = comp_size(G, c);
  if (!G->fsi_b) {
    bool ok = cudaMalloc(&G->fsi_b, 16 * sizeof(double)) == cudaSuccess;
    for (int c = 0; c < G->dim && ok; ++c) ok = cudaMalloc(&G->fsi_u[c], n[c] * es) == cudaSuccess;
    if (!ok) return set_error(FS_ERR_CUDA, "allocating the coupling workspace");
  }
  cudaStream_t s = G->stream;
  for (int c = 0; c < G->dim; ++c) cudaMemcpyAsync(G->fsi_u[c], st->u[c], n[c] * es, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(G->fsi_b, st->body, 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  T* u[3] = {(T*)st->u[0], (T*)st->u[1], (T*)(G->dim == 3 ? st->u[2] : nullptr)};
  T* us[3] = {(T*)G->ustar[0], (T*)G->ustar[1], (T*)G->ustar[2]};
  T* spec = (T*)G->spec;
  double* nb = G->fsi_b + 4;
  int k = 0;
  double xi = 0.0;
  while (k < G->fsi_iters) {
    if (k > 0)
      for (int c = 0; c < G->dim; ++c)
        cudaMemcpyAsync(st->u[c], G->fsi_u[c], n[c] * es, cudaMemcpyDeviceToDevice, s);
    ib_prepare<T>(G, st->body);
    launch_outflow_flux<T>(G, u);
    launch_predictor<T>(G, u, nullptr, us, dt, 0.0, 1.0, st->body);
    poisson_solve_from_velocity<T>(G, make_div_args<T>(G, us, st->body), spec);
    launch_correct<T>(G, us, spec, u);
    ib_forces<T>(G, st->body);
    cudaMemcpyAsync(nb, G->fsi_b, 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    body_rk4(G, nb, dt);
    FS_LAUNCH(G, "couple", couple_kernel<<<1, 32, 0, s>>>(st->body, nb, G->fsi_b + 8));
    ++k;
    cudaError_t e = cudaMemcpyAsync(&xi, G->fsi_b + 8, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(e, "fs_step (strong coupling)");
    if (!(xi == xi)) return set_error(FS_ERR_DIVERGED, "fs_step: NaN in the coupling iteration");
    if (xi < G->fsi_tol) break;
  }
  if (want_p) launch_to_pressure<T>(G, spec, st->p, G->rho / dt);
  G->fsi_last_iters = k;
  G->fsi_last_xi = xi;
  return FS_OK;
}

template int step_coupled<float>(fs_grid*, fs_state*, double, bool);
template int step_coupled<double>(fs_grid*, fs_state*, double, bool);

}  // namespace fs

using namespace fs;

template <>
Geom<double> fs_grid::geom<double>() const {
  Geom<double> g;
  g.dim = dim; g.nx = nx; g.ny = ny; g.nz = nz;
  for (int d = 0; d < 3; ++d) {
    g.per[d] = per[d];
    for (int s = 0; s < 2; ++s) {
      g.bc[d][s] = bc[d][s];
      for (int c = 0; c < 3; ++c) g.bcv[d][s][c] = bcv[d][s][c];
    }
  }
  g.hx = hx; g.hz = hz; g.ihx = 1.0 / hx; g.ihz = 1.0 / hz;
  g.ihy = ihy64; g.ihfy = ihfy64; g.thy = thy64;
  g.bforce = bforce.empty() ? nullptr : bf64;
  g.nu = nu;
  return g;
}

template <>
Geom<float> fs_grid::geom<float>() const {
  Geom<float> g;
  g.dim = dim; g.nx = nx; g.ny = ny; g.nz = nz;
  for (int d = 0; d < 3; ++d) {
    g.per[d] = per[d];
    for (int s = 0; s < 2; ++s) {
      g.bc[d][s] = bc[d][s];
      for (int c = 0; c < 3; ++c) g.bcv[d][s][c] = (float)bcv[d][s][c];
    }
  }
  g.hx = (float)hx; g.hz = (float)hz; g.ihx = (float)(1.0 / hx); g.ihz = (float)(1.0 / hz);
  g.ihy = ihy32; g.ihfy = ihfy32; g.thy = thy32;
  g.bforce = bforce.empty() ? nullptr : bf32;
  g.nu = (float)nu;
  return g;
}

extern "C" {

const char* fs_last_error(void) { return g_last_error.c_str(); }

int fs_create_grid(const fs_grid_desc* D, void* stream, fs_grid** out) {
  if (!D || !out) return set_error(FS_ERR_ARG, "fs_create_grid: NULL argument");
  *out = nullptr;
  if (D->dim != 2 && D->dim != 3) return set_error(FS_ERR_ARG, "dim must be 2 or 3");
  const int nz = D->dim == 3 ? D->n[2] : 1;
  if (D->n[0] < 2 || D->n[1] < 2 || nz < 1 || (D->dim == 3 && nz < 2))
    return set_error(FS_ERR_ARG, "cell counts must be >= 2");
  if (D->precision != FS_FP64 && D->precision != FS_MIXED) return set_error(FS_ERR_ARG, "unknown precision");
  if (D->conv_scheme != FS_CENTRAL2 && D->conv_scheme != FS_UPWIND1) return set_error(FS_ERR_ARG, "unknown convection scheme");
  if (D->time_scheme != FS_FE && D->time_scheme != FS_RK3) return set_error(FS_ERR_ARG, "unknown time scheme");
  fs_grid* G = new (std::nothrow) fs_grid();
  if (!G) return set_error(FS_ERR_ARG, "out of host memory");
  G->dim = D->dim;
  G->nx = D->n[0];
  G->ny = D->n[1];
  G->nz = nz;
  G->nu = D->nu;
  G->rho = D->rho > 0 ? D->rho : 1.0;
  G->conv = D->conv_scheme;
  G->scheme = D->time_scheme;
  G->prec = D->precision;
  G->stream = (cudaStream_t)stream;
  const int n[3] = {G->nx, G->ny, G->nz};
  for (int d = 0; d < 3; ++d) {
    for (int s = 0; s < 2; ++s) {
      G->bc[d][s] = d < D->dim ? D->bc[d][s] : FS_BC_PERIODIC;
      for (int c = 0; c < 3; ++c) G->bcv[d][s][c] = d < D->dim ? D->bc_val[d][s][c] : 0.0;
    }
    G->per[d] = G->bc[d][0] == FS_BC_PERIODIC;
    if ((G->bc[d][0] == FS_BC_PERIODIC) != (G->bc[d][1] == FS_BC_PERIODIC)) {
      delete G;
      return set_error(FS_ERR_ARG, "periodic boundary on one side only");
    }
    for (int s = 0; s < 2; ++s) {
      const int k = G->bc[d][s];
      if (k < FS_BC_PERIODIC || k > FS_BC_OUTFLOW || (k == FS_BC_INFLOW && (d != 0 || s != 0)) ||
          (k == FS_BC_OUTFLOW && (d != 0 || s != 1))) {
        delete G;
        return set_error(FS_ERR_ARG, "inflow is x-low only, outflow x-high only");
      }
    }
    std::vector<double> xf(n[d] + 1);
    if (d < D->dim) {
      if (!D->xf[d]) {
        delete G;
        return set_error(FS_ERR_ARG, "missing face coordinates");
      }
      for (int i = 0; i <= n[d]; ++i) xf[i] = D->xf[d][i];
    } else {
      xf = {0.0, 1.0};
    }
    std::vector<double> h(n[d]), xc(n[d]), hf(n[d] + 1), th(n[d] + 1, 0.5);
    for (int i = 0; i < n[d]; ++i) {
      h[i] = xf[i + 1] - xf[i];
      xc[i] = 0.5 * (xf[i] + xf[i + 1]);
      if (!(h[i] > 0)) {
        delete G;
        return set_error(FS_ERR_ARG, "face coordinates must increase");
      }
    }
    const double L = xf[n[d]] - xf[0];
    if (G->per[d]) {
      for (int f = 0; f < n[d]; ++f) {
        const double xl = f > 0 ? xc[f - 1] : xc[n[d] - 1] - L;
        hf[f] = xc[f] - xl;
        th[f] = (xf[f] - xl) / hf[f];
      }
      hf[n[d]] = hf[0];
      th[n[d]] = th[0];
    } else {
      for (int f = 1; f < n[d]; ++f) {
        hf[f] = xc[f] - xc[f - 1];
        th[f] = (xf[f] - xc[f - 1]) / hf[f];
      }
      hf[0] = h[0];
      hf[n[d]] = h[n[d] - 1];
    }
    G->xf[d] = xf;
    G->h[d] = h;
    G->hf[d] = hf;
    G->th[d] = th;
  }
  if (!uniform(G->h[0]) || (G->dim == 3 && !uniform(G->h[2]))) {
    delete G;
    return set_error(FS_ERR_ARG, "x and z spacing must be uniform (transform directions)");
  }
  if (G->per[1] && !uniform(G->h[1])) {
    delete G;
    return set_error(FS_ERR_ARG, "a periodic y direction must be uniform");
  }
  if (G->dim == 3 && (!G->per[0] || !G->per[2])) {
    delete G;
    return set_error(FS_ERR_UNSUPPORTED, "3-D grids need periodic x and z");
  }
  if ((G->per[0] && G->nx % 2) || (G->dim == 3 && G->nz % 2)) {
    delete G;
    return set_error(FS_ERR_ARG, "periodic transform directions need an even cell count");
  }
  if (G->scheme == FS_RK3 && !G->per[0] && G->bc[0][1] == FS_BC_OUTFLOW) {
    delete G;
    return set_error(FS_ERR_UNSUPPORTED, "RK3 is provided for grids without an outflow");
  }
  G->hx = G->h[0][0];
  G->hz = G->h[2][0];
  G->xmode = G->per[0] ? 0 : 1;
  G->yspec = G->per[1];
  if (!factorize(G->nx, G->px) || (G->dim == 3 && !factorize(G->nz, G->pz)) ||
      (G->yspec && !factorize(G->ny, G->py))) {
    delete G;
    return set_error(FS_ERR_UNSUPPORTED, "transform length with a prime factor > 13");
  }
  if ((double)(G->nx + 1) * (G->ny + 1) * (G->nz + 1) >= 2147483647.0) {
    delete G;
    return set_error(FS_ERR_UNSUPPORTED, "fields of 2^31 or more elements (32-bit kernel indexing)");
  }
  if (G->yspec && 2ull * (G->ny + 1) * 2 * elem_size(G) > 200 * 1024) {
    delete G;
    return set_error(FS_ERR_UNSUPPORTED, "periodic ny too large for one slot pair's line in shared memory");
  }
  if (!G->yspec && (size_t)G->ny * 32 * 8 > 200 * 1024) {
    delete G;
    return set_error(FS_ERR_UNSUPPORTED, "ny too large for the shared-memory tridiagonal staging (max 800)");
  }
  if (D->body_force) G->bforce.assign(D->body_force, D->body_force + G->ny);

  // device metrics
  const int ny = G->ny;
  std::vector<double> ihy(ny), ihfy(ny + 1), thy(ny + 1);
  for (int j = 0; j < ny; ++j) ihy[j] = 1.0 / G->h[1][j];
  for (int j = 0; j <= ny; ++j) {
    ihfy[j] = 1.0 / G->hf[1][j];
    thy[j] = G->th[1][j];
  }
  bool ok = upload(&G->ihy64, ihy) == cudaSuccess && upload(&G->ihfy64, ihfy) == cudaSuccess &&
            upload(&G->thy64, thy) == cudaSuccess && upload(&G->ihy32, cast<float>(ihy)) == cudaSuccess &&
            upload(&G->ihfy32, cast<float>(ihfy)) == cudaSuccess && upload(&G->thy32, cast<float>(thy)) == cudaSuccess &&
            upload(&G->hy64, G->h[1]) == cudaSuccess && upload(&G->hfy64, G->hf[1]) == cudaSuccess;
  for (int d = 0; d < 3 && ok; ++d) ok = upload(&G->xf64[d], G->xf[d]) == cudaSuccess;
  if (ok && !G->bforce.empty())
    ok = upload(&G->bf64, G->bforce) == cudaSuccess && upload(&G->bf32, cast<float>(G->bforce)) == cudaSuccess;
  // workspaces
  const size_t es = elem_size(G);
  for (int c = 0; c < G->dim && ok; ++c) {
    ok = cudaMalloc(&G->ustar[c], comp_size(G, c) * es) == cudaSuccess;
    if (ok && G->scheme == FS_RK3) ok = cudaMalloc(&G->ustage[c], comp_size(G, c) * es) == cudaSuccess;
  }
  const size_t cells = (size_t)G->nx * G->ny * G->nz;
  if (ok) ok = cudaMalloc(&G->spec, cells * std::max(es, sizeof(double))) == cudaSuccess;
  if (ok) ok = dalloc(&G->scal, 64) == cudaSuccess && cudaMemset(G->scal, 0, 64 * sizeof(double)) == cudaSuccess;
  if (ok) ok = dalloc(&G->red, 64) == cudaSuccess;
  if (ok) ok = cudaMalloc(&G->dstatus, sizeof(unsigned)) == cudaSuccess &&
               cudaMemset(G->dstatus, 0, sizeof(unsigned)) == cudaSuccess;
  if (ok) ok = G->prec == FS_MIXED ? (make_twiddles<float>(G->px) == cudaSuccess &&
                                      (G->dim == 2 || make_twiddles<float>(G->pz) == cudaSuccess) &&
                                      (!G->yspec || make_twiddles<float>(G->py) == cudaSuccess))
                                   : (make_twiddles<double>(G->px) == cudaSuccess &&
                                      (G->dim == 2 || make_twiddles<double>(G->pz) == cudaSuccess) &&
                                      (!G->yspec || make_twiddles<double>(G->py) == cudaSuccess));
  if (ok) ok = cudaStreamCreateWithFlags(&G->ystream2, cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&G->yev[0], cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&G->yev[1], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    free_all(G);
    delete G;
    return set_error(FS_ERR_CUDA, "allocating grid workspaces");
  }
  int rc = build_tables(G);
  if (rc != FS_OK) {
    free_all(G);
    delete G;
    return rc;
  }
  *out = G;
  return FS_OK;
}

int fs_destroy_grid(fs_grid* G) {
  if (!G) return FS_OK;
  cudaStreamSynchronize(G->stream);
  for (cudaEvent_t e : G->prof_pool) cudaEventDestroy(e);
  free_adj_buffers(G->adj);
  free_ib3(G);
  free_all(G);
  delete G;
  return FS_OK;
}

int fs_set_stream(fs_grid* G, void* stream) {
  if (!G) return set_error(FS_ERR_ARG, "NULL grid");
  G->stream = (cudaStream_t)stream;
  return FS_OK;
}

int fs_field_extent(const fs_grid* G, int comp, int ext[3]) {
  if (!G || !ext) return set_error(FS_ERR_ARG, "NULL argument");
  if (comp < -1 || comp >= G->dim) return set_error(FS_ERR_ARG, "component out of range");
  const int n[3] = {G->nx, G->ny, G->nz};
  for (int d = 0; d < 3; ++d) ext[d] = n[d] + ((comp == d && !G->per[d]) ? 1 : 0);
  return FS_OK;
}

long long fs_kernel_launches(const fs_grid* G) { return G ? G->launches : 0; }

int fs_set_tuning(fs_grid* G, const char* key, int value) {
  if (!G || !key) return set_error(FS_ERR_ARG, "NULL argument");
  const std::string k(key);
  if (k == "stencil_bx") {
    if (value != 0 && value != 32 && value != 64 && value != 128 && value != 256)
      return set_error(FS_ERR_ARG, "stencil_bx must be 32, 64, 128 or 256");
    G->tune_stencil_bx = value;
  } else if (k == "fft_lines") {
    if (value < 0 || value > 16) return set_error(FS_ERR_ARG, "fft_lines must be in 1..16");
    G->tune_fft_lines = value;
  } else if (k == "predictor_cells") {
    if (value != 0 && value != 1 && value != 2 && value != 4)
      return set_error(FS_ERR_ARG, "predictor_cells must be 1, 2 or 4");
    G->tune_pred_vw = value;
  } else if (k == "predictor_zmarch") {
    if (value < 0 || value > 64) return set_error(FS_ERR_ARG, "predictor_zmarch must be in 0..64");
    G->tune_zmarch = value;
  } else if (k == "ysplit") {
    if (value != 0 && value != 1) return set_error(FS_ERR_ARG, "ysplit must be 0 or 1");
    G->tune_ysplit = value;
  } else if (k == "pdl") {
    if (value != 0 && value != 1) return set_error(FS_ERR_ARG, "pdl must be 0 or 1");
    G->use_pdl = value == 1;
  } else if (k == "predictor_staged") {
    if (value != 0 && value != 1) return set_error(FS_ERR_ARG, "predictor_staged must be 0 or 1");
    G->tune_staged = value == 1;
  } else if (k == "predictor_chunk") {
    if (value < -1 || value > G->nz) return set_error(FS_ERR_ARG, "predictor_chunk must be -1 .. nz");
    G->tune_pred_chunk = value;
  } else if (k == "y_spectral") {
    // periodic y: 1 (default) DFT along y in the field precision with the exact zero mode;
    // 0 the FP64 cyclic tridiagonal solve per x/z wavenumber (the wall-normal path)
    if (value != 0 && value != 1) return set_error(FS_ERR_ARG, "y_spectral must be 0 or 1");
    if (!G->per[1]) return value == 1 ? FS_OK : set_error(FS_ERR_ARG, "y_spectral applies to a periodic y");
    if ((value == 1) == (G->yspec != 0)) return FS_OK;
    if (value == 0 && (size_t)G->ny * 32 * 8 > 200 * 1024)
      return set_error(FS_ERR_UNSUPPORTED, "ny too large for the shared-memory tridiagonal staging (max 800)");
    const cudaError_t e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return cuda_check(e, "fs_set_tuning");
    free_ytables(G);
    if (G->lamy) cudaFree(G->lamy);
    if (G->lamxz) cudaFree(G->lamxz);
    G->lamy = G->lamxz = nullptr;
    G->yspec = value;
    return build_tables(G);
  } else if (k == "ysolve_segments") {
    if (value != 0 && value != 4 && value != 8 && value != 16)
      return set_error(FS_ERR_ARG, "ysolve_segments must be 4, 8 or 16");
    if (value == G->tune_ynseg) return FS_OK;
    G->tune_ynseg = value;
    if (G->yspec) return FS_OK;   // periodic y has no partitioned solve
    const cudaError_t e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return cuda_check(e, "fs_set_tuning");
    free_ytables(G);
    return build_tables(G);
  } else if (k == "ysolve_twist_columns") {
    if (value != 0 && value != 32 && value != 64)
      return set_error(FS_ERR_ARG, "ysolve_twist_columns must be 0, 32 or 64");
    if (value == G->tune_ytw_cols) return FS_OK;
    G->tune_ytw_cols = value;
    if (G->yspec) return FS_OK;
    const cudaError_t e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return cuda_check(e, "fs_set_tuning");
    free_ytables(G);
    return build_tables(G);
  } else if (k == "xz_plane") {
    if (value < 0 || value > 2) return set_error(FS_ERR_ARG, "xz_plane must be 0, 1 or 2");
    G->tune_xzplane = value;
  } else if (k == "ysolve_tiled") {
    if (value != 0 && value != 1) return set_error(FS_ERR_ARG, "ysolve_tiled must be 0 or 1");
    G->tune_ytile = value == 1;
  } else if (k == "ysolve_twisted") {
    if (value < -1 || value > 1) return set_error(FS_ERR_ARG, "ysolve_twisted must be -1, 0 or 1");
    if (value == G->tune_ytwist) return FS_OK;
    G->tune_ytwist = value;
    if (G->yspec) return FS_OK;
    const cudaError_t e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return cuda_check(e, "fs_set_tuning");
    free_ytables(G);
    return build_tables(G);
  } else {
    return set_error(FS_ERR_ARG, "unknown tuning key " + k);
  }
  return FS_OK;
}

int fs_device_status(fs_grid* G, unsigned* bits) {
  if (!G || !bits) return set_error(FS_ERR_ARG, "NULL argument");
  cudaError_t e = cudaMemcpyAsync(bits, G->dstatus, sizeof(unsigned), cudaMemcpyDeviceToHost, G->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(G->dstatus, 0, sizeof(unsigned), G->stream);
  if (e != cudaSuccess) return cuda_check(e, "fs_device_status");
  return FS_OK;
}

int fs_profile_begin(fs_grid* G, const char* filter) {
  if (!G) return set_error(FS_ERR_ARG, "NULL grid");
  G->prof_on = true;
  G->prof_filter = filter ? filter : "";
  G->prof_used = 0;
  G->prof_names.clear();
  return FS_OK;
}

int fs_profile_end(fs_grid* G, char* report, int len) {
  if (!G) return set_error(FS_ERR_ARG, "NULL grid");
  G->prof_on = false;
  cudaError_t e = cudaStreamSynchronize(G->stream);
  if (e != cudaSuccess) return cuda_check(e, "fs_profile_end");
  std::vector<std::string> names;
  std::vector<long long> count;
  std::vector<double> total;
  for (size_t r = 0; r < G->prof_names.size(); ++r) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, G->prof_pool[2 * r], G->prof_pool[2 * r + 1]);
    size_t q = 0;
    while (q < names.size() && names[q] != G->prof_names[r]) ++q;
    if (q == names.size()) {
      names.push_back(G->prof_names[r]);
      count.push_back(0);
      total.push_back(0.0);
    }
    count[q] += 1;
    total[q] += ms;
  }
  std::string out;
  char line[256];
  for (size_t q = 0; q < names.size(); ++q) {
    snprintf(line, sizeof(line), "%s %lld %.6f\n", names[q].c_str(), count[q], total[q]);
    out += line;
  }
  if (report && len > 0) {
    strncpy(report, out.c_str(), (size_t)len - 1);
    report[len - 1] = 0;
  }
  G->prof_used = 0;
  G->prof_names.clear();
  return FS_OK;
}

int fs_set_ib_markers(fs_grid* G, const fs_body_desc* b) {
  if (!G || !b) return set_error(FS_ERR_ARG, "NULL argument");
  if (G->dim != 2) return set_error(FS_ERR_UNSUPPORTED, "immersed bodies are provided for 2-D grids");
  if (G->scheme != FS_FE) return set_error(FS_ERR_UNSUPPORTED, "immersed bodies use forward Euler");
  if (b->nm < 3 || !b->X0 || !b->Y0 || !b->ds) return set_error(FS_ERR_ARG, "need >= 3 markers with X0, Y0, ds");
  if (!uniform(G->h[1])) return set_error(FS_ERR_ARG, "immersed bodies need uniform y spacing");
  if (b->delta_kernel != FS_PESKIN4 && b->delta_kernel != FS_ROMA3) return set_error(FS_ERR_ARG, "unknown delta kernel");
  free_body(G);
  IBDev& B = G->ib;
  B.nm = b->nm;
  B.kernel = b->delta_kernel;
  B.centre[0] = b->centre[0];
  B.centre[1] = b->centre[1];
  B.omega = b->omega;
  B.mass = b->mass;
  B.k = b->stiffness;
  B.c = b->damping;
  B.active[0] = b->active[0];
  B.active[1] = b->active[1];
  // contours: vertex m is joined to nxt[m] (each contour closes on its first vertex)
  const int nm = b->nm;
  std::vector<int> nxt(nm);
  {
    std::vector<int> starts;
    if (b->ncontour > 1) {
      if (!b->contour_start) return set_error(FS_ERR_ARG, "ncontour > 1 needs contour_start");
      starts.assign(b->contour_start, b->contour_start + b->ncontour);
    } else {
      starts.push_back(0);
    }
    if (starts[0] != 0) return set_error(FS_ERR_ARG, "the first contour must start at marker 0");
    for (size_t k = 0; k < starts.size(); ++k) {
      const int a = starts[k], e = k + 1 < starts.size() ? starts[k + 1] : nm;
      if (e - a < 3 || e > nm) return set_error(FS_ERR_ARG, "contours need increasing starts and >= 3 markers each");
      for (int m = a; m < e; ++m) nxt[m] = m + 1 < e ? m + 1 : a;
    }
  }
  // bounding box with a margin so the early-out never decides a point near an edge
  double xmin = b->X0[0], xmax = b->X0[0], ymin = b->Y0[0], ymax = b->Y0[0];
  for (int m = 0; m < nm; ++m) {
    xmin = std::min(xmin, b->X0[m]);
    xmax = std::max(xmax, b->X0[m]);
    ymin = std::min(ymin, b->Y0[m]);
    ymax = std::max(ymax, b->Y0[m]);
  }
  const double mg = 1e-6 * (std::fabs(xmax - xmin) + std::fabs(ymax - ymin) + 1.0);
  B.poly_bb[0] = xmin - mg;
  B.poly_bb[1] = xmax + mg;
  B.poly_bb[2] = ymin - mg;
  B.poly_bb[3] = ymax + mg;
  // edges sorted by their lowest point (a row at height y is crossed only by edges whose lowest
  // point lies in [y - ehmax, y])
  std::vector<int> eo(nm);
  for (int m = 0; m < nm; ++m) eo[m] = m;
  auto elo = [&](int m) { return std::min(b->Y0[m], b->Y0[nxt[m]]); };
  std::stable_sort(eo.begin(), eo.end(), [&](int p, int q) { return elo(p) < elo(q); });
  std::vector<double> EAX(nm), EAY(nm), EBX(nm), EBY(nm), EY0(nm);
  B.ehmax = 0.0;
  for (int k = 0; k < nm; ++k) {
    const int a = eo[k], c = nxt[a];
    EAX[k] = b->X0[a];
    EAY[k] = b->Y0[a];
    EBX[k] = b->X0[c];
    EBY[k] = b->Y0[c];
    EY0[k] = elo(a);
    B.ehmax = std::max(B.ehmax, std::max(b->Y0[a], b->Y0[c]) - EY0[k]);
  }
  // bins of the sorted edges over their lowest y, one grid spacing high
  {
    B.ebin0 = EY0[0];
    B.ebinh = G->h[1][0];
    B.nebin = (int)std::ceil((EY0[nm - 1] - EY0[0]) / B.ebinh) + 1;
    if (B.nebin > (1 << 26)) return set_error(FS_ERR_ARG, "the body's edges span too many rows");
  }
  std::vector<int> ebin((size_t)B.nebin + 1, nm);
  {
    int k = 0;
    for (int b = 0; b <= B.nebin; ++b) {
      const double lo = B.ebin0 + b * B.ebinh;
      while (k < nm && EY0[k] < lo) ++k;
      ebin[b] = k;
    }
  }
  // markers sorted by the cell that holds their rest position (row-major), and the cell bins
  const double x0 = G->xf[0][0], y0 = G->xf[1][0], hy = G->h[1][0];
  std::vector<long long> ci(nm), cj(nm);
  long long cimin = 0, cimax = 0, cjmin = 0, cjmax = 0;
  for (int m = 0; m < nm; ++m) {
    ci[m] = (long long)std::floor((b->X0[m] - x0) / G->hx);
    cj[m] = (long long)std::floor((b->Y0[m] - y0) / hy);
    cimin = m ? std::min(cimin, ci[m]) : ci[m];
    cimax = m ? std::max(cimax, ci[m]) : ci[m];
    cjmin = m ? std::min(cjmin, cj[m]) : cj[m];
    cjmax = m ? std::max(cjmax, cj[m]) : cj[m];
  }
  if ((cimax - cimin + 1) * (cjmax - cjmin + 1) > (1LL << 28))
    return set_error(FS_ERR_ARG, "the body's markers span more than 2^28 cells");
  B.bx0 = (int)cimin;
  B.by0 = (int)cjmin;
  B.nbx = (int)(cimax - cimin + 1);
  B.nby = (int)(cjmax - cjmin + 1);
  auto key = [&](int m) { return (cj[m] - cjmin) * B.nbx + (ci[m] - cimin); };
  std::vector<int> order(nm);
  for (int m = 0; m < nm; ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return key(p) < key(q); });
  std::vector<double> X(nm), Y(nm), S(nm);
  for (int m = 0; m < nm; ++m) {
    X[m] = b->X0[order[m]];
    Y[m] = b->Y0[order[m]];
    S[m] = b->ds[order[m]];
  }
  std::vector<int> bins((size_t)B.nbx * B.nby + 1, 0);
  {
    size_t k = 0;
    for (size_t cell = 0; cell <= (size_t)B.nbx * B.nby; ++cell) {
      while (k < (size_t)nm && (size_t)key(order[k]) < cell) ++k;
      bins[cell] = (int)k;
    }
  }
  // grid units of the sorted markers (the cells of the bins above)
  std::vector<int2> GI(nm);
  std::vector<double> GF(2 * (size_t)nm), REL(2 * (size_t)nm);
  for (int m = 0; m < nm; ++m) {
    GI[m] = make_int2((int)ci[order[m]], (int)cj[order[m]]);
    GF[2 * m] = (X[m] - x0) / G->hx - (double)ci[order[m]];
    GF[2 * m + 1] = (Y[m] - y0) / hy - (double)cj[order[m]];
    REL[2 * m] = X[m] - b->centre[0];
    REL[2 * m + 1] = Y[m] - b->centre[1];
  }
  B.horder = order;
  bool ok = upload(&B.gi, GI) == cudaSuccess;
  std::vector<double> DSH(nm);
  for (int m = 0; m < nm; ++m) DSH[m] = S[m] * G->hx;
  if (G->prec == FS_MIXED) {
    float *gf = nullptr, *rel = nullptr, *dsh = nullptr;
    ok = ok && upload(&gf, cast<float>(GF)) == cudaSuccess && upload(&rel, cast<float>(REL)) == cudaSuccess &&
         upload(&dsh, cast<float>(DSH)) == cudaSuccess;
    B.gf = gf;
    B.rel = rel;
    B.dsh = dsh;
  } else {
    double *gf = nullptr, *rel = nullptr, *dsh = nullptr;
    ok = ok && upload(&gf, GF) == cudaSuccess && upload(&rel, REL) == cudaSuccess && upload(&dsh, DSH) == cudaSuccess;
    B.gf = gf;
    B.rel = rel;
    B.dsh = dsh;
  }
  ok = ok && cudaMalloc(&B.wfac, 2 * (size_t)nm * elem_size(G)) == cudaSuccess;
  ok = ok && upload(&B.X0, X) == cudaSuccess && upload(&B.Y0, Y) == cudaSuccess && upload(&B.ds, S) == cudaSuccess &&
            upload(&B.EAX, EAX) == cudaSuccess && upload(&B.EAY, EAY) == cudaSuccess &&
            upload(&B.EBX, EBX) == cudaSuccess && upload(&B.EBY, EBY) == cudaSuccess &&
            upload(&B.EY0, EY0) == cudaSuccess && upload(&B.order, order) == cudaSuccess &&
            upload(&B.bin_start, bins) == cudaSuccess && upload(&B.ebin, ebin) == cudaSuccess;
  {
    const size_t nf = comp_size(G, 0) + comp_size(G, 1);
    if (ok) ok = dalloc(&B.iblist, nf) == cudaSuccess && dalloc(&B.ibcount, 1) == cudaSuccess &&
                 cudaMemset(B.ibcount, 0, sizeof(unsigned)) == cudaSuccess;
  }
  const size_t es = elem_size(G);
  for (int c = 0; c < 2 && ok; ++c) {
    const size_t n = comp_size(G, c);
    ok = dalloc(&B.flags[c], n) == cudaSuccess && cudaMalloc(&B.num[c], n * es) == cudaSuccess &&
         cudaMalloc(&B.den[c], n * es) == cudaSuccess && cudaMalloc(&B.f[c], n * es) == cudaSuccess &&
         cudaMemset(B.num[c], 0, n * es) == cudaSuccess && cudaMemset(B.den[c], 0, n * es) == cudaSuccess &&
         cudaMemset(B.flags[c], 0, n) == cudaSuccess && cudaMemset(B.f[c], 0, n * es) == cudaSuccess;
  }
  if (ok) ok = dalloc(&B.part, 3 * (size_t)((2 * b->nm * 16 + 255) / 256)) == cudaSuccess;
  if (ok) ok = dalloc(&B.fn, 2 * b->nm) == cudaSuccess && dalloc(&B.q, 2 * b->nm) == cudaSuccess &&
               dalloc(&B.F, 4) == cudaSuccess && cudaMemset(B.F, 0, 4 * sizeof(double)) == cudaSuccess &&
               dalloc(&B.ticket, 1) == cudaSuccess && cudaMemset(B.ticket, 0, sizeof(unsigned)) == cudaSuccess;
  if (!ok) {
    free_body(G);
    return set_error(FS_ERR_CUDA, "allocating immersed-body buffers");
  }
  G->has_body = true;
  return FS_OK;
}

int fs_step(fs_grid* G, fs_state* st, double dt, int nsteps) {
  if (!G || !st) return set_error(FS_ERR_ARG, "NULL argument");
  for (int c = 0; c < G->dim; ++c)
    if (!st->u[c]) return set_error(FS_ERR_ARG, "NULL velocity component");
  if (G->has_body && !st->body) return set_error(FS_ERR_ARG, "a grid with a body needs st->body");
  if (nsteps < 0) return set_error(FS_ERR_ARG, "nsteps < 0");
  for (int s = 0; s < nsteps; ++s) {
    double h = dt;
    if (dt <= 0) {
      double d[3];
      int rc = fs_diagnostics(G, st, d);
      if (rc != FS_OK) return rc;
      if (!std::isfinite(d[0]) || !std::isfinite(d[2])) return set_error(FS_ERR_DIVERGED, "non-finite velocity");
      double hmin = G->hx;
      for (double v : G->h[1]) hmin = std::min(hmin, v);
      if (G->dim == 3) hmin = std::min(hmin, G->hz);
      h = 0.5 * hmin / std::max(d[0], 1e-30);
    }
    const bool want_p = st->p && s == nsteps - 1;
    if (G->has_body && G->fsi_iters > 1 && G->ib.mass > 0) {
      const int rc = G->prec == FS_MIXED ? step_coupled<float>(G, st, h, want_p) : step_coupled<double>(G, st, h, want_p);
      if (rc != FS_OK) return rc;
      continue;
    }
    if (G->prec == FS_MIXED) step_once<float>(G, st, h, want_p);
    else step_once<double>(G, st, h, want_p);
  }
  return cuda_check(cudaGetLastError(), "fs_step launch");
}

namespace {
int step_adjoint_entry(fs_grid* G, const fs_state* st_n, fs_state* lam, const double* dJdF, bool dJdF_dev,
                       fs_param_grad* g, double dt) {
  if (!G || !st_n || !lam) return set_error(FS_ERR_ARG, "NULL argument");
  if (!(dt > 0)) return set_error(FS_ERR_ARG, "the adjoint needs the fixed step dt > 0 of the forward step");
  for (int c = 0; c < G->dim; ++c)
    if (!st_n->u[c] || !lam->u[c]) return set_error(FS_ERR_ARG, "NULL velocity component");
  if (G->has_body) {
    if (!st_n->body || !lam->body) return set_error(FS_ERR_ARG, "a grid with a body needs st_n->body and lam->body");
    if (G->ib.omega != 0.0)
      return set_error(FS_ERR_UNSUPPORTED, "adjoint of a body with a prescribed surface rotation");
  }
  if (G->les_cs > 0.0) return set_error(FS_ERR_UNSUPPORTED, "adjoint of a step with the Smagorinsky model");
  if (G->has_ib3) return set_error(FS_ERR_UNSUPPORTED, "adjoint of a grid with a static 3-D box body");
  if (G->has_body && G->fsi_iters > 1 && G->ib.mass > 0)
    return G->prec == FS_MIXED ? step_adjoint_coupled<float>(G, st_n, lam, dJdF, dJdF_dev, g, dt)
                               : step_adjoint_coupled<double>(G, st_n, lam, dJdF, dJdF_dev, g, dt);
  return G->prec == FS_MIXED ? step_adjoint<float>(G, st_n, lam, dJdF, g, dt, nullptr, nullptr, dJdF_dev)
                             : step_adjoint<double>(G, st_n, lam, dJdF, g, dt, nullptr, nullptr, dJdF_dev);
}
}  // namespace

int fs_step_adjoint(fs_grid* G, const fs_state* st_n, fs_state* lam, const double* dJdF, fs_param_grad* g,
                    double dt) {
  return step_adjoint_entry(G, st_n, lam, dJdF, false, g, dt);
}

int fs_step_adjoint_dev(fs_grid* G, const fs_state* st_n, fs_state* lam, const double* dJdF, fs_param_grad* g,
                        double dt) {
  return step_adjoint_entry(G, st_n, lam, dJdF, true, g, dt);
}

namespace {
int check_recordable(const fs_grid* G, void* const* v1, void* const* v2) {
  if (!v1 || !v2) return set_error(FS_ERR_ARG, "NULL stage arrays");
  for (int c = 0; c < G->dim; ++c)
    if (!v1[c] || !v2[c]) return set_error(FS_ERR_ARG, "NULL stage component");
  if (G->scheme != FS_RK3) return set_error(FS_ERR_ARG, "stage states exist for the RK3 scheme only");
  if (G->has_body || G->has_ib3) return set_error(FS_ERR_UNSUPPORTED, "recorded stages of a grid with a body");
  if (G->les_cs > 0.0) return set_error(FS_ERR_UNSUPPORTED, "recorded stages with the Smagorinsky model");
  return FS_OK;
}
}  // namespace

int fs_step_record(fs_grid* G, fs_state* st, double dt, void* const* v1, void* const* v2) {
  if (!G || !st) return set_error(FS_ERR_ARG, "NULL argument");
  for (int c = 0; c < G->dim; ++c)
    if (!st->u[c]) return set_error(FS_ERR_ARG, "NULL velocity component");
  if (!(dt > 0)) return set_error(FS_ERR_ARG, "a recorded step needs a fixed dt > 0");
  int rc = check_recordable(G, v1, v2);
  if (rc != FS_OK) return rc;
  if (G->prec == FS_MIXED) step_once<float>(G, st, dt, st->p != nullptr, v1, v2);
  else step_once<double>(G, st, dt, st->p != nullptr, v1, v2);
  return cuda_check(cudaGetLastError(), "fs_step_record launch");
}

int fs_step_adjoint_recorded(fs_grid* G, const fs_state* st_n, void* const* v1, void* const* v2, fs_state* lam,
                             fs_param_grad* g, double dt) {
  if (!G || !st_n || !lam) return set_error(FS_ERR_ARG, "NULL argument");
  if (!(dt > 0)) return set_error(FS_ERR_ARG, "the adjoint needs the fixed step dt > 0 of the forward step");
  for (int c = 0; c < G->dim; ++c)
    if (!st_n->u[c] || !lam->u[c]) return set_error(FS_ERR_ARG, "NULL velocity component");
  int rc = check_recordable(G, v1, v2);
  if (rc != FS_OK) return rc;
  return G->prec == FS_MIXED ? step_adjoint<float>(G, st_n, lam, nullptr, g, dt, v1, v2)
                             : step_adjoint<double>(G, st_n, lam, nullptr, g, dt, v1, v2);
}

int fs_solve_pressure(fs_grid* G, const double* rhs, double* p) {
  if (!G || !rhs || !p) return set_error(FS_ERR_ARG, "NULL argument");
  const size_t cells = (size_t)G->nx * G->ny * G->nz;
  if (G->prec == FS_MIXED) {
    return set_error(FS_ERR_UNSUPPORTED, "fs_solve_pressure takes FP64 data; use an FS_FP64 grid");
  }
  if (p != rhs) {
    cudaError_t e = cudaMemcpyAsync(p, rhs, cells * sizeof(double), cudaMemcpyDeviceToDevice, G->stream);
    if (e != cudaSuccess) return cuda_check(e, "fs_solve_pressure copy");
  }
  poisson_solve_inplace<double>(G, p);
  return cuda_check(cudaGetLastError(), "fs_solve_pressure launch");
}

namespace fs {
__global__ void bf_convert_kernel(const double* __restrict__ src, double* __restrict__ d64, float* __restrict__ d32,
                                  int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    d64[t] = src[t];
    d32[t] = (float)src[t];
  }
}
}  // namespace fs

int fs_set_body_force(fs_grid* G, const double* fx) {
  if (!G || !fx) return set_error(FS_ERR_ARG, "NULL argument");
  if (G->bforce.empty()) return set_error(FS_ERR_STATE, "the grid was created without a body_force profile");
  FS_LAUNCH(G, "set_body_force", bf_convert_kernel<<<(G->ny + 127) / 128, 128, 0, G->stream>>>(fx, G->bf64, G->bf32, G->ny));
  return cuda_check(cudaGetLastError(), "fs_set_body_force");
}

int fs_set_coupling(fs_grid* G, int max_subiters, double tol) {
  if (!G) return set_error(FS_ERR_ARG, "NULL grid");
  if (max_subiters < 1 || !(tol > 0.0)) return set_error(FS_ERR_ARG, "fs_set_coupling: max_subiters >= 1, tol > 0");
  G->fsi_iters = max_subiters;
  G->fsi_tol = tol;
  return FS_OK;
}

int fs_set_les(fs_grid* G, double cs) {
  if (!G) return set_error(FS_ERR_ARG, "NULL grid");
  if (!(cs >= 0.0)) return set_error(FS_ERR_ARG, "fs_set_les: C_s must be >= 0");
  if (cs > 0.0) {
    if (G->dim != 3 || !G->per[0] || !G->per[1] || !G->per[2])
      return set_error(FS_ERR_UNSUPPORTED, "the Smagorinsky model is provided for 3-D grids periodic in x, y and z");
    if (G->conv != FS_CENTRAL2 || G->has_body || G->has_ib3)
      return set_error(FS_ERR_UNSUPPORTED, "the Smagorinsky model is provided for central convection without bodies");
    if (!G->les_nu[0]) {
      const size_t n = (size_t)G->nx * G->ny * G->nz * elem_size(G);
      for (int q = 0; q < 4; ++q)
        if (cudaMalloc(&G->les_nu[q], n) != cudaSuccess) return set_error(FS_ERR_CUDA, "allocating nu_t");
    }
  }
  G->les_cs = cs;
  return FS_OK;
}

int fs_ib_face_count(fs_grid* G, int* count) {
  if (!G || !count) return set_error(FS_ERR_ARG, "NULL argument");
  if (!G->has_body) return set_error(FS_ERR_STATE, "no 2-D body attached");
  unsigned n = 0;
  cudaError_t e = cudaMemcpyAsync(&n, G->ib.ibcount, sizeof(unsigned), cudaMemcpyDeviceToHost, G->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
  if (e != cudaSuccess) return cuda_check(e, "fs_ib_face_count");
  *count = (int)n;
  return FS_OK;
}

int fs_coupling_stats(const fs_grid* G, int* subiters, double* xi) {
  if (!G) return set_error(FS_ERR_ARG, "NULL grid");
  if (subiters) *subiters = G->fsi_last_iters;
  if (xi) *xi = G->fsi_last_xi;
  return FS_OK;
}

int fs_set_stiffness(fs_grid* G, double k) {
  if (!G) return set_error(FS_ERR_ARG, "NULL grid");
  if (!G->has_body) return set_error(FS_ERR_STATE, "no body attached");
  G->ib.k = k;
  return FS_OK;
}

int fs_forces_device(fs_grid* G, double* F) {
  if (!G || !F) return set_error(FS_ERR_ARG, "NULL argument");
  if (G->has_ib3)
    return cuda_check(cudaMemcpyAsync(F, G->ib3.F, 3 * sizeof(double), cudaMemcpyDeviceToDevice, G->stream),
                      "fs_forces_device");
  if (!G->has_body) return set_error(FS_ERR_STATE, "no body attached");
  return cuda_check(cudaMemcpyAsync(F, G->ib.F, 3 * sizeof(double), cudaMemcpyDeviceToDevice, G->stream),
                    "fs_forces_device");
}

int fs_forces(fs_grid* G, double* F, double* torque, double* q) {
  if (!G) return set_error(FS_ERR_ARG, "NULL grid");
  if (G->has_ib3) {
    if (!G->ib3.have_forces) return set_error(FS_ERR_STATE, "no step has run with the box body");
    double h[3];
    cudaError_t e = cudaMemcpyAsync(h, G->ib3.F, 3 * sizeof(double), cudaMemcpyDeviceToHost, G->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return cuda_check(e, "fs_forces");
    if (F)
      for (int d = 0; d < 3; ++d) F[d] = h[d];
    if (torque) *torque = 0.0;
    if (q) {
      const int nm = G->ib3.nm;
      std::vector<double> qs(3 * (size_t)nm);
      e = cudaMemcpy(qs.data(), G->ib3.q, qs.size() * sizeof(double), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_check(e, "fs_forces q");
      for (int m = 0; m < nm; ++m)
        for (int d = 0; d < 3; ++d) q[3 * (size_t)m + d] = qs[(size_t)d * nm + m];
    }
    return FS_OK;
  }
  if (!G->has_body || !G->ib.have_forces) return set_error(FS_ERR_STATE, "no FSI step has run");
  double h[4];
  cudaError_t e = cudaMemcpyAsync(h, G->ib.F, 3 * sizeof(double), cudaMemcpyDeviceToHost, G->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
  if (e != cudaSuccess) return cuda_check(e, "fs_forces");
  if (F) {
    F[0] = h[0];
    F[1] = h[1];
  }
  if (torque) *torque = h[2];
  if (q) {
    std::vector<double> qs(2 * G->ib.nm);
    e = cudaMemcpy(qs.data(), G->ib.q, qs.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_check(e, "fs_forces q");
    for (int m = 0; m < G->ib.nm; ++m) {
      const int o = G->ib.horder[m];
      q[2 * o] = qs[2 * m];
      q[2 * o + 1] = qs[2 * m + 1];
    }
  }
  return FS_OK;
}

int fs_diagnostics(fs_grid* G, const fs_state* st, double out[3]) {
  if (!G || !st || !out) return set_error(FS_ERR_ARG, "NULL argument");
  double* d = G->scal + 16;
  if (G->prec == FS_MIXED) {
    float* u[3] = {(float*)st->u[0], (float*)st->u[1], (float*)st->u[2]};
    launch_diagnostics<float>(G, u, d);
  } else {
    double* u[3] = {(double*)st->u[0], (double*)st->u[1], (double*)st->u[2]};
    launch_diagnostics<double>(G, u, d);
  }
  cudaError_t e = cudaMemcpyAsync(out, d, 3 * sizeof(double), cudaMemcpyDeviceToHost, G->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
  return cuda_check(e, "fs_diagnostics");
}

}  // extern "C"
