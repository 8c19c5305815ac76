// Immersed-boundary and rigid-body kernels (§2.3.2-2.3.3 of the paper), 2-D bodies.
//
//   classify_solid   solid faces: crossing-number test of (face - w) against the
//                    rest contours, every FP64 operation rounded on its own
//                    (__d*_rn) so the integer decision is the oracle's bit for bit;
//                    one block per face row finds the edges crossing the row's
//                    height once (edges sorted by their lowest point, the candidates
//                    found by bisection), then every face of the row counts the
//                    crossings to its right (both components in one launch)
//   classify_ib      IB faces: non-solid faces with a solid same-component neighbour,
//                    appended to a list of the step's IB faces
//   ib_fn            F_N of Eq. (19) per marker and component (support nodes that are
//                    not solid): 16 lanes per (marker, component), one support node
//                    each, summed by shuffles
//   ib_gather        the normalised interpolation of Eq. (18) on each IB face: the
//                    markers of the cells around the face (markers binned by the cell of
//                    their rest position, visited row by row in a fixed order) are summed
//                    in FP64 registers, so every face has one writer, no atomics, and a
//                    bitwise reproducible result
//   ib_force         q_i of Eq. (20) per marker (FP64 sums, 16 lanes per marker and
//                    component); the last block to finish forms F = rho sum q_i dV_i and
//                    the torque in a fixed order (FP64) and, in a forward step, the
//                    Eq. (12) RK4 update of the body with the force frozen
//   rk4              the same body update on its own (coupling sub-iterations)
//
// Kernel evaluation: node offsets from markers are formed in FP64, the
// kernel phi in the field precision T.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fs_internal.cuh"

namespace fs {

namespace {

constexpr int kT = 256;

// Edges of the rest contours, sorted by their lowest y (ey0): edge k runs from (ax, ay)
// to (bx, by) in surface order.
struct Poly {
  const double* ax;
  const double* ay;
  const double* bx;
  const double* by;
  const double* ey0;
  int n;
  double hmax;     // largest edge height
  double bb[4];
  // edge bins: ybin[k] is the first edge whose lowest point is >= ybin0 + k / iybin (nybin + 1 entries)
  const int* ybin;
  double ybin0, iybin;
  int nybin;
  double ihx;      // 1 / h_x of the grid
};

__device__ __forceinline__ bool inside_polygon(const Poly& P, double px, double py) {
  if (px < P.bb[0] || px > P.bb[1] || py < P.bb[2] || py > P.bb[3]) return false;
  bool in = false;
  for (int e = 0; e < P.n; ++e) {
    const double ax = P.ax[e], ay = P.ay[e];
    const double bx = P.bx[e], by = P.by[e];
    if ((ay > py) != (by > py)) {
      const double xint = __dadd_rn(ax, __ddiv_rn(__dmul_rn(__dsub_rn(py, ay), __dsub_rn(bx, ax)), __dsub_rn(by, ay)));
      if (px < xint) in = !in;
    }
  }
  return in;
}

// face position of component c at storage index (i, j)
__device__ __forceinline__ void face_pos(int c, int i, int j, const double* xf, const double* yf, double& px,
                                         double& py) {
  if (c == 0) {
    px = xf[i];
    py = __dmul_rn(0.5, __dadd_rn(yf[j], yf[j + 1]));
  } else {
    px = __dmul_rn(0.5, __dadd_rn(xf[i], xf[i + 1]));
    py = yf[j];
  }
}

constexpr int kRowCross = 1024;   // crossings of one face row held in shared memory

struct Flags {
  uint8_t* p[2];
};

// grid (rows, 2 components); face rows outside the polygon's displaced box are cleared.
__global__ void __launch_bounds__(kT) classify_solid_kernel(Flags flags, int ex0, int ey0, int ex1, int ey1,
                                                             const double* __restrict__ xf,
                                                             const double* __restrict__ yf,
                                                             const double* __restrict__ body, Poly P,
                                                             unsigned* __restrict__ ibcount) {
  __shared__ double xs[kRowCross];
  __shared__ int xi[kRowCross];
  __shared__ int cnt, elo, ehi;
  const int c = blockIdx.y, j = blockIdx.x;
  if (j == 0 && c == 0 && threadIdx.x == 0) *ibcount = 0u;   // the step's IB face list starts empty
  const int ex = c ? ex1 : ex0, ey = c ? ey1 : ey0;
  if (j >= ey) return;
  uint8_t* row = (c ? flags.p[1] : flags.p[0]) + (size_t)j * ex;
  const double wx = body[0], wy = body[1];
  const double py = __dsub_rn(c == 0 ? __dmul_rn(0.5, __dadd_rn(yf[j], yf[j + 1])) : yf[j], wy);
  if (py < P.bb[2] || py > P.bb[3]) {
    for (int i = threadIdx.x; i < ex; i += blockDim.x) row[i] = 0;
    return;
  }
  // the face x of index i, minus the displacement, as the oracle forms it
  auto px_of = [&](int i) {
    return __dsub_rn(c == 0 ? xf[i] : __dmul_rn(0.5, __dadd_rn(xf[i], xf[i + 1])), wx);
  };
  if (threadIdx.x == 0) {
    cnt = 0;
    // only edges whose lowest point lies in [py - hmax, py] can cross the row: their range from the
    // edge bins (twice the largest height as the lower bound keeps a rounded height from excluding one)
    const double b0 = (py - 2.0 * P.hmax - P.ybin0) * P.iybin, b1 = (py - P.ybin0) * P.iybin;
    const int k0 = (int)fmin(fmax(floor(b0), 0.0), (double)P.nybin);
    const int k1 = (int)fmin(fmax(floor(b1) + 1.0, 0.0), (double)P.nybin);
    elo = P.ybin[k0];
    ehi = P.ybin[k1];
  }
  __syncthreads();
  // x where each edge crosses the row's height (the order of the crossings does not matter to the parity)
  for (int e = elo + threadIdx.x; e < ehi; e += blockDim.x) {
    const double ax = P.ax[e], ay = P.ay[e];
    const double bx = P.bx[e], by = P.by[e];
    if ((ay > py) != (by > py)) {
      const double xint = __dadd_rn(ax, __ddiv_rn(__dmul_rn(__dsub_rn(py, ay), __dsub_rn(bx, ax)), __dsub_rn(by, ay)));
      const int k = atomicAdd(&cnt, 1);
      if (k < kRowCross) xs[k] = xint;
    }
  }
  __syncthreads();
  const int nc = cnt;
  if (nc > kRowCross) {
    for (int i = threadIdx.x; i < ex; i += blockDim.x) row[i] = inside_polygon(P, px_of(i), py) ? 1 : 0;
    return;
  }
  // per crossing: the number of faces left of it (px < xint; px grows with i), from an estimate
  // corrected by exact comparisons; a face is solid when an odd number of crossings lie to its right
  int npow = 1;
  while (npow < nc) npow <<= 1;
  for (int k = threadIdx.x; k < npow; k += blockDim.x) {
    int idx = 0x7fffffff;
    if (k < nc) {
      const double xint = xs[k];
      const double x0 = c == 0 ? xf[0] : 0.5 * (xf[0] + xf[1]);
      const double gs = ceil((xint + wx - x0) * P.ihx);
      idx = (int)fmin(fmax(gs, 0.0), (double)ex);
      while (idx > 0 && !(px_of(idx - 1) < xint)) --idx;
      while (idx < ex && px_of(idx) < xint) ++idx;
    }
    xi[k] = idx;
  }
  __syncthreads();
  // bitonic sort of the npow entries (padding sorts last)
  for (int kk = 2; kk <= npow; kk <<= 1)
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < npow; i += blockDim.x) {
        const int l = i ^ jj;
        if (l > i) {
          const int a = xi[i], b = xi[l];
          if ((a > b) == ((i & kk) == 0)) {
            xi[i] = b;
            xi[l] = a;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < ex; i += blockDim.x) {
    // crossings with idx > i lie to the right of face i: nc - (first position with idx > i)
    int lo = 0, hi = nc;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (xi[mid] <= i) lo = mid + 1;
      else hi = mid;
    }
    row[i] = ((nc - lo) & 1) ? 1 : 0;
  }
}

// marks face t IB when it is not solid and a same-component neighbour is; returns that
__device__ __forceinline__ bool ib_face(uint8_t* __restrict__ flags, long long t, int ex, int ey, int perx,
                                        int pery) {
  const int i = (int)(t % ex), j = (int)(t / ex);
  const uint8_t me = flags[t];
  if (me & 1) return false;
  bool nb = false;
  const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int a = i + di[q], b = j + dj[q];
    if (a < 0 || a >= ex) {
      if (!perx) continue;
      a = a < 0 ? a + ex : a - ex;
    }
    if (b < 0 || b >= ey) {
      if (!pery) continue;
      b = b < 0 ? b + ey : b - ey;
    }
    nb = nb || (flags[(size_t)b * ex + a] & 1);
  }
  if (nb) flags[t] = me | 2;
  return nb;
}

// Block bx of nbx of the IB classification of component c; the IB faces are appended to list as
// (index << 1) | component (the list's order varies from run to run; nothing computed from it
// depends on the order)
// Only faces of the index box ilo..ihi x jlo..jhi (the body's displaced bounding box plus two faces)
// can be solid or next to a solid face.
__device__ __forceinline__ void classify_ib_block(Flags F, int ex0, int ey0, int ex1, int ey1, int perx, int pery,
                                                  unsigned* __restrict__ list, unsigned* __restrict__ count, int c,
                                                  int bx, int nbx, int ilo, int ihi, int jlo, int jhi) {
  const int ex = c ? ex1 : ex0, ey = c ? ey1 : ey0;
  uint8_t* __restrict__ flags = c ? F.p[1] : F.p[0];
  // (a periodic direction is visited whole: IB faces may sit across its seam)
  const int i0 = perx ? 0 : max(ilo, 0), i1 = perx ? ex - 1 : min(ihi, ex - 1);
  const int j0 = pery ? 0 : max(jlo, 0), j1 = pery ? ey - 1 : min(jhi, ey - 1);
  const int w = i1 - i0 + 1;
  const long long total = (w > 0 && j1 >= j0) ? (long long)w * (j1 - j0 + 1) : 0;
  const long long span = (long long)nbx * blockDim.x;
  for (long long t0 = (long long)bx * blockDim.x; t0 < total; t0 += span) {
    const long long tl = t0 + threadIdx.x;
    const long long t = tl < total ? (long long)(j0 + tl / w) * ex + (i0 + tl % w) : 0;
    bool isib = false;
    if (tl < total) isib = ib_face(flags, t, ex, ey, perx, pery);
    // warp-aggregated append
    const unsigned m = __ballot_sync(0xffffffffu, isib);
    if (m) {
      const int lane = threadIdx.x & 31;
      unsigned base = 0;
      if (lane == __ffs(m) - 1) base = atomicAdd(count, (unsigned)__popc(m));
      base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
      if (isib) list[base + __popc(m & ((1u << lane) - 1u))] = ((unsigned)t << 1) | (unsigned)c;
    }
  }
}

template <typename T>
__device__ __forceinline__ T phi_kernel(int kind, T r) {
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

struct IBGeom {
  int ex[2], ey[2];
  double x0c[2], y0c[2];   // position of node (0, 0) of each component
  double hx, hy;
  double ihx, ihy, ihxy;   // 1 / hx, 1 / hy, 1 / (hx hy)
  int kind;
  int width;               // support nodes per direction (3 Roma, 4 Peskin)
  const double* xf;
  const double* yf;
  const double* hyv;       // cell widths in y
  const double* hfyv;      // face spacings in y
  double hfx;              // uniform x spacing
};

// Markers in grid units.  A marker's rest position in cell units from the grid origin,
// g = (X0 - x0) / h, is held as an integer part gi = floor(g) and a fraction gf in [0, 1)
// (host-computed in FP64 when the body is attached, gf stored in the field precision T);
// the step's displacement in cell units, W = w / h, splits the same way.  The offset of a
// node from a marker in grid units, r = (node - X) / h, is then an integer difference plus a
// difference of fractions, formed in T: no FP64 arithmetic per node, which on B300's narrow
// FP64 pipe would bound every immersed-boundary kernel.  Node i of component c sits at
// (i + o_c) h from the origin: o = 0 along the component's own direction, 1/2 across.
template <typename T>
struct Shift {
  int wi[2];   // floor(W) per direction
  T wf[2];     // W - floor(W)
};

template <typename T>
__device__ __forceinline__ Shift<T> shift_of(const double* body, double ihx, double ihy) {
  Shift<T> S;
  const double W[2] = {body[0] * ihx, body[1] * ihy};
  for (int d = 0; d < 2; ++d) {
    const double f = floor(W[d]);
    S.wi[d] = (int)f;
    S.wf[d] = T(W[d] - f);
  }
  return S;
}

// first support node of a marker (integer part gi, fraction gf) along one direction for nodes at
// offset o, and the marker's position relative to that direction's node 0 as (sint, sfr)
template <typename T>
__device__ __forceinline__ int first_node_units(int kind, int gi, T gf, int wi, T wf, T o, int& sint, T& sfr) {
  T t = gf + wf - o;                 // in [-1/2, 2)
  const T k = floor(t);
  sint = gi + wi + (int)k;
  sfr = t - k;                       // in [0, 1)
  return kind == FS_PESKIN4 ? sint - 1 : sint + (int)floor(sfr + T(0.5)) - 1;
}

// The W x W support of a (marker, component) pair: first nodes (i0, j0) and the 1-D kernel
// weights of its W columns (px) and W rows (py), in the field precision.
template <typename T, int W>
__device__ __forceinline__ void support_of(const IBGeom& G, const Shift<T>& S, int2 mi, T gfx, T gfy, int c, int& i0,
                                           int& j0, T (&px)[W], T (&py)[W]) {
  int sx, sy;
  T fx, fy;
  i0 = first_node_units<T>(G.kind, mi.x, gfx, S.wi[0], S.wf[0], c ? T(0.5) : T(0), sx, fx);
  j0 = first_node_units<T>(G.kind, mi.y, gfy, S.wi[1], S.wf[1], c ? T(0) : T(0.5), sy, fy);
#pragma unroll
  for (int a = 0; a < W; ++a) {
    px[a] = phi_kernel<T>(G.kind, T(i0 + a - sx) - fx);
    py[a] = phi_kernel<T>(G.kind, T(j0 + a - sy) - fy);
  }
}

// the rest polygon's bounding box: xmin, xmax, ymin, ymax
struct Box4 {
  double v[4];
  __host__ __device__ double operator[](int i) const { return v[i]; }
};

// F_N_i of Eq. (19), one thread per (marker, component): delta_h summed over the support nodes
// that are not solid; stores the interpolation weight factor of Eq. (18),
// wfac = dV_i / (F_N_i h_x h_y) (then w_i(x) = phi phi wfac), with dsh = dV_i = ds_i h_x.
// F_N needs only the solid faces, so it runs in the same launch as the IB classification: blocks
// [0, 2 nbc) classify (component = block / nbc), the rest take F_N.
template <typename T, int W>
__global__ void __launch_bounds__(kT) ib_classify_fn_kernel(Flags flags, int ex0, int ey0, int ex1, int ey1,
                                                            int perx, int pery, unsigned* __restrict__ list,
                                                            unsigned* __restrict__ count, int nbc, const IBGeom G,
                                                            int nm, const int2* __restrict__ gi,
                                                            const T* __restrict__ gf, const T* __restrict__ dsh,
                                                            const double* __restrict__ body, T* __restrict__ wfac,
                                                            const Box4 bbox) {
  if ((int)blockIdx.x < 2 * nbc) {
    // the displaced bounding box in face indices (uniform spacing near the body), with a margin
    __shared__ int box[4];
    if (threadIdx.x == 0) {
      box[0] = (int)floor((bbox[0] + body[0] - G.xf[0]) * G.ihx) - 2;
      box[1] = (int)ceil((bbox[1] + body[0] - G.xf[0]) * G.ihx) + 2;
      box[2] = (int)floor((bbox[2] + body[1] - G.yf[0]) * G.ihy) - 2;
      box[3] = (int)ceil((bbox[3] + body[1] - G.yf[0]) * G.ihy) + 2;
    }
    __syncthreads();
    classify_ib_block(flags, ex0, ey0, ex1, ey1, perx, pery, list, count, blockIdx.x / nbc, blockIdx.x % nbc, nbc,
                      box[0], box[1], box[2], box[3]);
    return;
  }
  __shared__ Shift<T> S;
  if (threadIdx.x == 0) S = shift_of<T>(body, G.ihx, G.ihy);
  __syncthreads();
  const int pair = (blockIdx.x - 2 * nbc) * blockDim.x + threadIdx.x;
  if (pair >= 2 * nm) return;
  const int m = pair >> 1, c = pair & 1;
  int i0, j0;
  T px[W], py[W];
  support_of<T, W>(G, S, gi[m], gf[2 * m], gf[2 * m + 1], c, i0, j0, px, py);
  const uint8_t* fl = c ? flags.p[1] : flags.p[0];
  const int ex = G.ex[c], ey = G.ey[c];
  T s = T(0);
#pragma unroll
  for (int b = 0; b < W; ++b) {
    const int j = j0 + b;
    if (j < 0 || j >= ey) continue;
    T r = T(0);
#pragma unroll
    for (int a = 0; a < W; ++a) {
      const int i = i0 + a;
      if (i >= 0 && i < ex && !(fl[(size_t)j * ex + i] & 1)) r += px[a];   // solid nodes are left out of F_N
    }
    s += r * py[b];
  }
  wfac[pair] = s > T(0) ? dsh[m] / s : T(0);
}

// Marker bins of the rest positions (see IBDev): markers of cell (ci, cj) are the sorted
// markers [start[k], start[k + 1]), k = (cj - by0) nbx + (ci - bx0).
struct Bins {
  const int* start;
  int bx0, by0, nbx, nby;
  double x0, y0;   // grid origin (cell (0, 0) starts there)
};

// Eq. (18) in normalised form, one warp per IB face: u_IB = sum_i w_i v_i / sum_i w_i,
// w_i = delta_h(x - X_i) dV_i / F_N_i, over the markers whose support holds the face.  The face's
// rest-frame position x - w picks the rows of rest cells that can hold such a marker; within a
// row the markers of consecutive cells are one contiguous run of the sorted markers.  The runs
// of the (at most 5) rows are laid end to end and the warp's lanes take one marker each (all
// loads in flight at once), then the lanes' sums are reduced by shuffles in a fixed tree: one
// writer per face, no atomics, the same result on every run.
template <typename T, bool WARP>
__global__ void __launch_bounds__(kT) ib_gather_kernel(const IBGeom G, const Bins Bn, const int2* __restrict__ gi,
                                                       const T* __restrict__ gf, const T* __restrict__ rel,
                                                       const T* __restrict__ wfac, const double* __restrict__ body,
                                                       double omega, const unsigned* __restrict__ list,
                                                       const unsigned* __restrict__ count, T* num0, T* den0, T* num1,
                                                       T* den1) {
  __shared__ Shift<T> S;
  __shared__ T vbs[2];
  if (threadIdx.x == 0) {
    S = shift_of<T>(body, G.ihx, G.ihy);
    vbs[0] = T(body[2]);
    vbs[1] = T(body[3]);
  }
  __syncthreads();
  const unsigned n = *count;
  constexpr int reach = 2;   // cells on each side of the face's own that can hold a marker within the support
  const int lane = WARP ? (int)(threadIdx.x & 31) : 0;
  const unsigned stride = WARP ? (gridDim.x * blockDim.x) >> 5 : gridDim.x * blockDim.x;
  const unsigned first = WARP ? (blockIdx.x * blockDim.x + threadIdx.x) >> 5 : blockIdx.x * blockDim.x + threadIdx.x;
  for (unsigned e = first; e < n; e += stride) {
    const unsigned code = list[e];
    const int c = (int)(code & 1u);
    const size_t f = code >> 1;
    const int i = (int)(f % (size_t)G.ex[c]), j = (int)(f / (size_t)G.ex[c]);
    // the face's offsets from a marker with (gi, gf): (i - gi - wi) + (ox - gf - wf), likewise in y
    const int ai = i - S.wi[0], aj = j - S.wi[1];
    const T afx = (c ? T(0.5) : T(0)) - S.wf[0], afy = (c ? T(0) : T(0.5)) - S.wf[1];
    // rest cells that can hold a marker with |face - marker| < 2 cells (Peskin) or 1.5 (Roma): a marker
    // left out at the rounded window's edge would sit where the kernel vanishes
    const int fcx = ai + (int)floor(afx), fcy = aj + (int)floor(afy);
    const int ci0 = max(fcx - reach, Bn.bx0), ci1 = min(fcx + reach, Bn.bx0 + Bn.nbx - 1);
    const int cj0 = max(fcy - reach, Bn.by0), cj1 = min(fcy + reach, Bn.by0 + Bn.nby - 1);
    int roff[2 * reach + 1], rm0[2 * reach + 1];   // every row's run: offset in the candidate list, first marker
    int total = 0;
    if constexpr (WARP) {
      // lane r < 2 reach + 1: the run of row cj0 + r
      int m0 = 0, len = 0;
      if (lane <= 2 * reach && cj0 + lane <= cj1 && ci0 <= ci1) {
        const int row = (cj0 + lane - Bn.by0) * Bn.nbx - Bn.bx0;
        m0 = Bn.start[row + ci0];
        len = Bn.start[row + ci1 + 1] - m0;
      }
      // runs end to end: start offset of each row's run
      int off = len;
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
      }
      total = __shfl_sync(0xffffffffu, off, 2 * reach);
      off -= len;                                   // exclusive
#pragma unroll
      for (int q = 0; q <= 2 * reach; ++q) {
        roff[q] = __shfl_sync(0xffffffffu, off, q);
        rm0[q] = __shfl_sync(0xffffffffu, m0, q);
      }
    } else {
#pragma unroll
      for (int q = 0; q <= 2 * reach; ++q) {
        int m0 = 0, len = 0;
        if (cj0 + q <= cj1 && ci0 <= ci1) {
          const int row = (cj0 + q - Bn.by0) * Bn.nbx - Bn.bx0;
          m0 = Bn.start[row + ci0];
          len = Bn.start[row + ci1 + 1] - m0;
        }
        roff[q] = total;
        rm0[q] = m0;
        total += len;
      }
    }
    T num = T(0), den = T(0);
    const T vb = vbs[c];
    for (int k = lane; k < total; k += WARP ? 32 : 1) {
      // the row holding candidate k (empty rows have the next row's offset and are passed over)
      int m = rm0[0] + k;
#pragma unroll
      for (int q = 1; q <= 2 * reach; ++q)
        if (k >= roff[q]) m = rm0[q] + (k - roff[q]);
      const int2 mi = gi[m];
      const T rx = T(ai - mi.x) + (afx - gf[2 * m]);
      const T ry = T(aj - mi.y) + (afy - gf[2 * m + 1]);
      const T d = phi_kernel<T>(G.kind, rx) * phi_kernel<T>(G.kind, ry);
      const T wf = wfac[2 * m + c];
      if (d != T(0) && wf > T(0)) {
        const T w = d * wf;
        // marker velocity: body translation plus surface rotation (rel: rest position - centre)
        const T vm = omega == 0.0 ? vb : (c == 0 ? vb - T(omega) * rel[2 * m + 1] : vb + T(omega) * rel[2 * m]);
        num += w * vm;
        den += w;
      }
    }
    if constexpr (WARP) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
      }
    }
    if (lane == 0) {
      (c ? num1 : num0)[f] = num;
      (c ? den1 : den0)[f] = den;
    }
  }
}

// Eq. (12) with F frozen over the step: classical RK4 per active DOF (one thread).
__device__ void rk4_body(double* __restrict__ st, const double* __restrict__ F, double m, double k, double c, int ax,
                         int ay, double dt) {
  const int act[2] = {ax, ay};
  for (int d = 0; d < 2; ++d) {
    double w = st[d], v = st[2 + d];
    if (!act[d]) {
      st[d] = 0.0;
      st[2 + d] = 0.0;
      continue;
    }
    const double f = F[d];
    auto acc = [&](double x, double u) { return (f - c * u - k * x) / m; };
    const double k1x = v, k1v = acc(w, v);
    const double k2x = v + 0.5 * dt * k1v, k2v = acc(w + 0.5 * dt * k1x, v + 0.5 * dt * k1v);
    const double k3x = v + 0.5 * dt * k2v, k3v = acc(w + 0.5 * dt * k2x, v + 0.5 * dt * k2v);
    const double k4x = v + dt * k3v, k4v = acc(w + dt * k3x, v + dt * k3v);
    st[d] = w + dt / 6.0 * (k1x + 2.0 * k2x + 2.0 * k3x + k4x);
    st[2 + d] = v + dt / 6.0 * (k1v + 2.0 * k2v + 2.0 * k3v + k4v);
  }
}

__global__ void rk4_kernel(double* __restrict__ st, const double* __restrict__ F, double m, double k, double c,
                           int ax, int ay, double dt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) rk4_body(st, F, m, k, c, ax, ay, dt);
}

struct BodyODE {
  double* st;   // body state to advance after the force, or null
  double m, k, c, dt;
  int ax, ay;
};

// q_i = - sum_x f(x) delta_h(x - X_i) dv(x)   (Eq. 20), one thread per (marker, component), in
// the field precision (the grid is uniform near the body, so dv / (h_x h_y) = 1); then
// F = rho sum_i q_i dV_i and the torque rho sum_i dV_i (r_i x q_i) in FP64: each block sums its
// pairs' terms in a fixed tree into its slot of part, and the block that finishes last (the others
// publish their slot before taking a ticket; no block waits) sums the slots in a fixed order and,
// when asked, takes the body ODE step with that force.
template <typename T, int W>
__global__ void __launch_bounds__(kT) force_kernel(const IBGeom G, int nm, const int2* __restrict__ gi,
                                                   const T* __restrict__ gf, const T* __restrict__ rel,
                                                   const T* __restrict__ dsh, const double* body,
                                                   const T* __restrict__ f0, const T* __restrict__ f1, double rho,
                                                   double* __restrict__ q, double* __restrict__ part,
                                                   double* __restrict__ F, unsigned* __restrict__ ticket,
                                                   const BodyODE ode) {
  __shared__ Shift<T> S;
  __shared__ double s0[kT / 32], s1[kT / 32], s2[kT / 32];
  __shared__ bool last;
  if (threadIdx.x == 0) S = shift_of<T>(body, G.ihx, G.ihy);
  __syncthreads();
  const int pair = blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, b = 0.0, tq = 0.0;
  if (pair < 2 * nm) {
    const int m = pair >> 1, c = pair & 1;
    int i0, j0;
    T px[W], py[W];
    support_of<T, W>(G, S, gi[m], gf[2 * m], gf[2 * m + 1], c, i0, j0, px, py);
    const T* f = c ? f1 : f0;
    const int ex = G.ex[c], ey = G.ey[c];
    T sum = T(0);
#pragma unroll
    for (int bb = 0; bb < W; ++bb) {
      const int j = j0 + bb;
      if (j < 0 || j >= ey) continue;
      T r = T(0);
#pragma unroll
      for (int aa = 0; aa < W; ++aa) {
        const int i = i0 + aa;
        if (i >= 0 && i < ex) r += f[(size_t)j * ex + i] * px[aa];
      }
      sum += r * py[bb];
    }
    const T qv = -sum;
    q[pair] = (double)qv;
    // this pair's terms of F and of the torque (r = rest position - centre: the body only translates)
    const T dV = dsh[m];
    const T t = c == 0 ? -dV * rel[2 * m + 1] * qv : dV * rel[2 * m] * qv;
    (c == 0 ? a : b) = (double)(qv * dV);
    tq = (double)t;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    tq += __shfl_down_sync(0xffffffffu, tq, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s0[threadIdx.x >> 5] = a;
    s1[threadIdx.x >> 5] = b;
    s2[threadIdx.x >> 5] = tq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0, st = 0.0;
    for (int w = 0; w < kT / 32; ++w) {
      sa += s0[w];
      sb += s1[w];
      st += s2[w];
    }
    part[3 * blockIdx.x] = sa;
    part[3 * blockIdx.x + 1] = sb;
    part[3 * blockIdx.x + 2] = st;
  }
  // the last block to finish reduces the block sums
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  a = b = tq = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    a += __ldcg(part + 3 * k);
    b += __ldcg(part + 3 * k + 1);
    tq += __ldcg(part + 3 * k + 2);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    tq += __shfl_down_sync(0xffffffffu, tq, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    s0[threadIdx.x >> 5] = a;
    s1[threadIdx.x >> 5] = b;
    s2[threadIdx.x >> 5] = tq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0, st = 0.0;
    for (int w = 0; w < kT / 32; ++w) {
      sa += s0[w];
      sb += s1[w];
      st += s2[w];
    }
    F[0] = rho * sa;
    F[1] = rho * sb;
    F[2] = rho * st;
    *ticket = 0u;
    if (ode.st) rk4_body(ode.st, F, ode.m, ode.k, ode.c, ode.ax, ode.ay, ode.dt);
  }
}

IBGeom make_geom(const fs_grid* G) {
  IBGeom g;
  for (int c = 0; c < 2; ++c) {
    g.ex[c] = G->nx + ((c == 0 && !G->per[0]) ? 1 : 0);
    g.ey[c] = G->ny + ((c == 1 && !G->per[1]) ? 1 : 0);
  }
  g.hx = G->hx;
  g.hy = G->h[1][0];
  g.ihx = 1.0 / g.hx;
  g.ihy = 1.0 / g.hy;
  g.ihxy = 1.0 / (g.hx * g.hy);
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
  g.hfx = G->hx;
  return g;
}

}  // namespace

template <typename T>
void ib_prepare(fs_grid* G, const double* body_state) {
  IBDev& B = G->ib;
  Poly P;
  P.ax = B.EAX;
  P.ay = B.EAY;
  P.bx = B.EBX;
  P.by = B.EBY;
  P.ey0 = B.EY0;
  P.n = B.nm;
  P.hmax = B.ehmax;
  for (int q = 0; q < 4; ++q) P.bb[q] = B.poly_bb[q];
  P.ybin = B.ebin;
  P.ybin0 = B.ebin0;
  P.iybin = 1.0 / B.ebinh;
  P.nybin = B.nebin;
  P.ihx = 1.0 / G->hx;
  Flags dflags;
  dflags.p[0] = B.flags[0];
  dflags.p[1] = B.flags[1];
  int ex[2], ey[2];
  for (int c = 0; c < 2; ++c) {
    ex[c] = G->nx + ((c == 0 && !G->per[0]) ? 1 : 0);
    ey[c] = G->ny + ((c == 1 && !G->per[1]) ? 1 : 0);
  }
  FS_LAUNCH(G, "classify_solid", classify_solid_kernel<<<dim3(std::max(ey[0], ey[1]), 2), kT, 0, G->stream>>>(
                                     dflags, ex[0], ey[0], ex[1], ey[1], G->xf64[0], G->xf64[1], body_state, P,
                                     B.ibcount));
  const IBGeom g = make_geom(G);
  Box4 bbox;
  for (int q = 0; q < 4; ++q) bbox.v[q] = B.poly_bb[q];
  {
    // faces in the body's bounding box (plus margins), which the kernel visits
    const double bw = (B.poly_bb[1] - B.poly_bb[0]) / G->hx + 6.0, bh = (B.poly_bb[3] - B.poly_bb[2]) / G->h[1][0] + 6.0;
    const long long all = (long long)std::max(ex[0] * ey[0], ex[1] * ey[1]);
    const long long n = (G->per[0] || G->per[1]) ? all : std::min(all, (long long)(bw * bh) + 1);
    int nbc = (int)((n + kT - 1) / kT);
    if (nbc > 148 * 8) nbc = 148 * 8;
    const int nb = 2 * nbc + (2 * B.nm + kT - 1) / kT;
    if (g.width == 4)
      FS_LAUNCH(G, "classify_ib_fn", ib_classify_fn_kernel<T, 4><<<nb, kT, 0, G->stream>>>(
                                         dflags, ex[0], ey[0], ex[1], ey[1], G->per[0], G->per[1], B.iblist,
                                         B.ibcount, nbc, g, B.nm, B.gi, (const T*)B.gf, (const T*)B.dsh, body_state,
                                         (T*)B.wfac, bbox));
    else
      FS_LAUNCH(G, "classify_ib_fn", ib_classify_fn_kernel<T, 3><<<nb, kT, 0, G->stream>>>(
                                         dflags, ex[0], ey[0], ex[1], ey[1], G->per[0], G->per[1], B.iblist,
                                         B.ibcount, nbc, g, B.nm, B.gi, (const T*)B.gf, (const T*)B.dsh, body_state,
                                         (T*)B.wfac, bbox));
  }
  Bins bn{B.bin_start, B.bx0, B.by0, B.nbx, B.nby, G->xf[0][0], G->xf[1][0]};
  // IB faces: about two per marker and component.  Small bodies take a warp per face (the candidate
  // markers' loads all in flight: latency), large ones a thread per face (throughput); the kernel
  // strides over the list
  const bool warp = 4LL * B.nm * 32 <= 148LL * 2048;
  const int nb = (int)std::min<long long>(148LL * 8, (4LL * B.nm * (warp ? 32 : 1) + kT - 1) / kT + 1);
  if (warp)
    FS_LAUNCH(G, "ib_gather", ib_gather_kernel<T, true><<<nb, kT, 0, G->stream>>>(
                                  g, bn, B.gi, (const T*)B.gf, (const T*)B.rel, (const T*)B.wfac, body_state, B.omega,
                                  B.iblist, B.ibcount, (T*)B.num[0], (T*)B.den[0], (T*)B.num[1], (T*)B.den[1]));
  else
    FS_LAUNCH(G, "ib_gather", ib_gather_kernel<T, false><<<nb, kT, 0, G->stream>>>(
                                  g, bn, B.gi, (const T*)B.gf, (const T*)B.rel, (const T*)B.wfac, body_state, B.omega,
                                  B.iblist, B.ibcount, (T*)B.num[0], (T*)B.den[0], (T*)B.num[1], (T*)B.den[1]));
}

template <typename T>
void ib_forces(fs_grid* G, double* body_state, double* advance, double dt) {
  IBDev& B = G->ib;
  const IBGeom g = make_geom(G);
  BodyODE ode{nullptr, B.mass, B.k, B.c, dt, B.active[0], B.active[1]};
  if (advance && B.mass > 0) ode.st = advance;
  const int npb = (2 * B.nm + kT - 1) / kT;
  if (g.width == 4)
    FS_LAUNCH(G, "ib_force", force_kernel<T, 4><<<npb, kT, 0, G->stream>>>(
                                 g, B.nm, B.gi, (const T*)B.gf, (const T*)B.rel, (const T*)B.dsh, body_state,
                                 (const T*)B.f[0], (const T*)B.f[1], G->rho, B.q, B.part, B.F, B.ticket, ode));
  else
    FS_LAUNCH(G, "ib_force", force_kernel<T, 3><<<npb, kT, 0, G->stream>>>(
                                 g, B.nm, B.gi, (const T*)B.gf, (const T*)B.rel, (const T*)B.dsh, body_state,
                                 (const T*)B.f[0], (const T*)B.f[1], G->rho, B.q, B.part, B.F, B.ticket, ode));
  B.have_forces = true;
}

void body_rk4(fs_grid* G, double* body_state, double dt) {
  IBDev& B = G->ib;
  if (B.mass <= 0) return;
  FS_LAUNCH(G, "rk4", rk4_kernel<<<1, 32, 0, G->stream>>>(body_state, B.F, B.mass, B.k, B.c, B.active[0], B.active[1], dt));
}

template void ib_prepare<float>(fs_grid*, const double*);
template void ib_prepare<double>(fs_grid*, const double*);
template void ib_forces<float>(fs_grid*, double*, double*, double);
template void ib_forces<double>(fs_grid*, double*, double*, double);

}  // namespace fs
