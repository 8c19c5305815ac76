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
};

// first edge whose lowest point is >= v (or > v when strict)
__device__ __forceinline__ int edge_bound(const Poly& P, double v, bool strict) {
  int lo = 0, hi = P.n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const double e = P.ey0[mid];
    if (strict ? e <= v : e < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

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
                                                             const double* __restrict__ body, Poly P) {
  __shared__ double xs[kRowCross];
  __shared__ int cnt;
  const int c = blockIdx.y, j = blockIdx.x;
  const int ex = c ? ex1 : ex0, ey = c ? ey1 : ey0;
  if (j >= ey) return;
  uint8_t* row = (c ? flags.p[1] : flags.p[0]) + (size_t)j * ex;
  const double wx = body[0], wy = body[1];
  const double py = __dsub_rn(c == 0 ? __dmul_rn(0.5, __dadd_rn(yf[j], yf[j + 1])) : yf[j], wy);
  if (py < P.bb[2] || py > P.bb[3]) {
    for (int i = threadIdx.x; i < ex; i += blockDim.x) row[i] = 0;
    return;
  }
  __shared__ int elo, ehi;
  if (threadIdx.x == 0) {
    cnt = 0;
    // only edges whose lowest point lies in [py - hmax, py] can cross the row (twice the largest
    // height as the lower bound keeps a rounded edge height from excluding one)
    elo = edge_bound(P, py - 2.0 * P.hmax, false);
    ehi = edge_bound(P, py, true);
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
  for (int i = threadIdx.x; i < ex; i += blockDim.x) {
    const double px = __dsub_rn(c == 0 ? xf[i] : __dmul_rn(0.5, __dadd_rn(xf[i], xf[i + 1])), wx);
    bool in = false;
    if (nc > kRowCross) {
      in = inside_polygon(P, px, py);
    } else if (px >= P.bb[0] && px <= P.bb[1]) {
      for (int k = 0; k < nc; ++k)
        if (px < xs[k]) in = !in;
    }
    row[i] = in ? 1 : 0;
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

// grid (blocks, 2 components); the IB faces are appended to list as (index << 1) | component
// (the list's order varies from run to run; nothing computed from it depends on the order)
__global__ void classify_ib_kernel(Flags F, int ex0, int ey0, int ex1, int ey1, int perx, int pery,
                                   unsigned* __restrict__ list, unsigned* __restrict__ count) {
  const int c = blockIdx.y;
  const int ex = c ? ex1 : ex0, ey = c ? ey1 : ey0;
  uint8_t* __restrict__ flags = c ? F.p[1] : F.p[0];
  const long long total = (long long)ex * ey;
  const long long span = (long long)gridDim.x * blockDim.x;
  for (long long t0 = (long long)blockIdx.x * blockDim.x; t0 < total; t0 += span) {
    const long long t = t0 + threadIdx.x;
    bool isib = false;
    if (t < total) isib = ib_face(flags, t, ex, ey, perx, pery);
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

// first support node along one direction for marker coordinate X
__device__ __forceinline__ int first_node(const IBGeom& G, double X, double x0, double h) {
  const double s = (X - x0) / h;
  return G.kind == FS_PESKIN4 ? (int)floor(s) - 1 : (int)floor(s + 0.5) - 1;
}

__device__ __forceinline__ double node_x(const IBGeom& G, int c, int i) {
  return c == 0 ? G.xf[i] : __dmul_rn(0.5, __dadd_rn(G.xf[i], G.xf[i + 1]));
}
__device__ __forceinline__ double node_y(const IBGeom& G, int c, int j) {
  return c == 1 ? G.yf[j] : __dmul_rn(0.5, __dadd_rn(G.yf[j], G.yf[j + 1]));
}

// Support node of one lane: 16 lanes per (marker, component) pair, lane l -> node
// (a, b) = (l mod width, l / width); lanes with b >= width hold no node.
struct Lane {
  int pair, m, c, a, b;
  bool live;
};

__device__ __forceinline__ Lane lane_of(const IBGeom& G, int nm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  Lane L;
  L.pair = t >> 4;
  const int l = t & 15;
  L.m = L.pair >> 1;
  L.c = L.pair & 1;
  L.a = l % G.width;
  L.b = l / G.width;
  L.live = L.pair < 2 * nm;
  return L;
}

__device__ __forceinline__ double sum16(double s) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// F_N_i of Eq. (19): the 16 lanes of a (marker, component) pair evaluate delta_h at
// their support node and sum it over the nodes that are not solid by shuffles.
template <typename T>
__global__ void ib_fn_kernel(const IBGeom G, int nm, const double* __restrict__ X0, const double* __restrict__ Y0,
                             const double* __restrict__ body, const Flags flags, double* __restrict__ fn) {
  const Lane L = lane_of(G, nm);
  double s = 0.0;
  if (L.live && L.b < G.width) {
    const int c = L.c;
    const double X = X0[L.m] + body[0];
    const double Y = Y0[L.m] + body[1];
    const int i = first_node(G, X, G.x0c[c], G.hx) + L.a, j = first_node(G, Y, G.y0c[c], G.hy) + L.b;
    if (i >= 0 && i < G.ex[c] && j >= 0 && j < G.ey[c]) {
      const size_t f = (size_t)j * G.ex[c] + i;
      const uint8_t fl = (c ? flags.p[1] : flags.p[0])[f];
      const T py = phi_kernel<T>(G.kind, T((node_y(G, c, j) - Y) * G.ihy));
      const T px = phi_kernel<T>(G.kind, T((node_x(G, c, i) - X) * G.ihx));
      if (!(fl & 1)) s = (double)(px * py) * G.ihxy;   // solid nodes are excluded from F_N
    }
  }
  const double F = sum16(s);
  if (L.live && (threadIdx.x & 15) == 0) fn[L.pair] = F;
}

// Marker bins of the rest positions (see IBDev): markers of cell (ci, cj) are the sorted
// markers [start[k], start[k + 1]), k = (cj - by0) nbx + (ci - bx0).
struct Bins {
  const int* start;
  int bx0, by0, nbx, nby;
  double x0, y0;   // grid origin (cell (0, 0) starts there)
};

// Eq. (18) in normalised form on one IB face per thread: u_IB = sum_i w_i v_i / sum_i w_i,
// w_i = delta_h(x - X_i) dV_i / F_N_i, over the markers whose support holds the face.  The face's
// rest-frame position x - w picks the cells whose markers can reach it (the kernel's support
// plus one cell on each side); within a cell row the markers of consecutive cells are one
// contiguous run of the sorted markers, visited in order.  FP64 sums, one writer per face.
template <typename T>
__global__ void __launch_bounds__(kT) ib_gather_kernel(const IBGeom G, const Bins Bn, const double* __restrict__ X0,
                                                       const double* __restrict__ Y0, const double* __restrict__ ds,
                                                       const double* __restrict__ fn,
                                                       const double* __restrict__ body, double omega, double cx,
                                                       double cy, const unsigned* __restrict__ list,
                                                       const unsigned* __restrict__ count, T* num0, T* den0, T* num1,
                                                       T* den1) {
  const unsigned n = *count;
  const double wx = body[0], wy = body[1];
  const double reach = G.kind == FS_PESKIN4 ? 2.0 : 1.5;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const unsigned code = list[e];
    const int c = (int)(code & 1u);
    const size_t f = code >> 1;
    const int i = (int)(f % (size_t)G.ex[c]), j = (int)(f / (size_t)G.ex[c]);
    const double xf = node_x(G, c, i), yf = node_y(G, c, j);
    const double sx = (xf - wx - Bn.x0) * G.ihx, sy = (yf - wy - Bn.y0) * G.ihy;
    const int ci0 = max((int)floor(sx - reach) - 1, Bn.bx0), ci1 = min((int)floor(sx + reach) + 1, Bn.bx0 + Bn.nbx - 1);
    const int cj0 = max((int)floor(sy - reach) - 1, Bn.by0), cj1 = min((int)floor(sy + reach) + 1, Bn.by0 + Bn.nby - 1);
    double num = 0.0, den = 0.0;
    for (int cj = cj0; cj <= cj1 && ci0 <= ci1; ++cj) {
      const int row = (cj - Bn.by0) * Bn.nbx - Bn.bx0;
      const int m0 = Bn.start[row + ci0], m1 = Bn.start[row + ci1 + 1];
      for (int m = m0; m < m1; ++m) {
        const double X = X0[m] + wx, Y = Y0[m] + wy;
        const T py = phi_kernel<T>(G.kind, T((yf - Y) * G.ihy));
        const T px = phi_kernel<T>(G.kind, T((xf - X) * G.ihx));
        const T d = px * py;
        const double F = fn[2 * m + c];
        if (d == T(0) || !(F > 0.0)) continue;
        const T w = T((double)d * G.ihxy * (ds[m] * G.hx) / F);
        // marker velocity: body translation plus surface rotation
        const double vm = c == 0 ? body[2] - omega * (Y - (cy + wy)) : body[3] + omega * (X - (cx + wx));
        num += (double)(w * T(vm));
        den += (double)w;
      }
    }
    (c ? num1 : num0)[f] = T(num);
    (c ? den1 : den0)[f] = T(den);
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

// q_i = - sum_x f(x) delta_h(x - X_i) dv(x)   (Eq. 20), 16 lanes per marker and
// component; then F = rho sum_i q_i dV_i and the torque rho sum_i dV_i (r_i x q_i): each
// block sums its markers' terms (a fixed tree) into its slot of part, and the block that
// finishes last (the others publish their slot before taking a ticket; no block waits) sums
// the slots in a fixed order and, when asked, takes the body ODE step with that force.
template <typename T>
__global__ void __launch_bounds__(kT) force_kernel(const IBGeom G, int nm, const double* __restrict__ X0,
                                                   const double* __restrict__ Y0, const double* __restrict__ ds,
                                                   const double* body, const T* __restrict__ f0,
                                                   const T* __restrict__ f1, double cx, double cy, double rho,
                                                   double* __restrict__ q, double* __restrict__ part,
                                                   double* __restrict__ F, unsigned* __restrict__ ticket,
                                                   const BodyODE ode) {
  const Lane L = lane_of(G, nm);
  double s = 0.0, X = 0.0, Y = 0.0;
  if (L.live) {
    X = X0[L.m] + body[0];
    Y = Y0[L.m] + body[1];
  }
  if (L.live && L.b < G.width) {
    const int c = L.c;
    const T* f = c == 0 ? f0 : f1;
    const int i = first_node(G, X, G.x0c[c], G.hx) + L.a, j = first_node(G, Y, G.y0c[c], G.hy) + L.b;
    if (i >= 0 && i < G.ex[c] && j >= 0 && j < G.ey[c]) {
      const T py = phi_kernel<T>(G.kind, T((node_y(G, c, j) - Y) * G.ihy));
      const T px = phi_kernel<T>(G.kind, T((node_x(G, c, i) - X) * G.ihx));
      const double dvy = c == 0 ? G.hyv[j] : G.hfyv[j];
      s = (double)f[(size_t)j * G.ex[c] + i] * ((double)(px * py) * G.ihxy) * (G.hfx * dvy);
    }
  }
  s = sum16(s);
  // this pair's terms of F and the torque (held by the pair's first lane)
  __shared__ double s0[kT], s1[kT], s2[kT];
  double a = 0.0, b = 0.0, tq = 0.0;
  if (L.live && (threadIdx.x & 15) == 0) {
    const double qv = -s;
    q[L.pair] = qv;
    const double dV = ds[L.m] * G.hx;
    const double rx = X - (cx + body[0]), ry = Y - (cy + body[1]);
    if (L.c == 0) {
      a = qv * dV;
      tq = -dV * ry * qv;
    } else {
      b = qv * dV;
      tq = dV * rx * qv;
    }
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  s2[threadIdx.x] = tq;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = s0[0];
    part[3 * blockIdx.x + 1] = s1[0];
    part[3 * blockIdx.x + 2] = s2[0];
  }
  // the last block to finish reduces the block sums
  __shared__ bool last;
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
  __syncthreads();
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  s2[threadIdx.x] = tq;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    F[0] = rho * s0[0];
    F[1] = rho * s1[0];
    F[2] = rho * s2[0];
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
  Flags dflags;
  dflags.p[0] = B.flags[0];
  dflags.p[1] = B.flags[1];
  int ex[2], ey[2];
  for (int c = 0; c < 2; ++c) {
    ex[c] = G->nx + ((c == 0 && !G->per[0]) ? 1 : 0);
    ey[c] = G->ny + ((c == 1 && !G->per[1]) ? 1 : 0);
  }
  FS_LAUNCH(G, "classify_solid", classify_solid_kernel<<<dim3(std::max(ey[0], ey[1]), 2), kT, 0, G->stream>>>(
                                     dflags, ex[0], ey[0], ex[1], ey[1], G->xf64[0], G->xf64[1], body_state, P));
  cudaMemsetAsync(B.ibcount, 0, sizeof(unsigned), G->stream);
  {
    const long long n = (long long)std::max(ex[0] * ey[0], ex[1] * ey[1]);
    int nb = (int)((n + kT - 1) / kT);
    if (nb > 148 * 8) nb = 148 * 8;
    FS_LAUNCH(G, "classify_ib", classify_ib_kernel<<<dim3(nb, 2), kT, 0, G->stream>>>(
                                    dflags, ex[0], ey[0], ex[1], ey[1], G->per[0], G->per[1], B.iblist, B.ibcount));
  }
  const IBGeom g = make_geom(G);
  const int nlane = 2 * B.nm * 16;
  FS_LAUNCH(G, "ib_fn", ib_fn_kernel<T><<<(nlane + kT - 1) / kT, kT, 0, G->stream>>>(g, B.nm, B.X0, B.Y0, body_state,
                                                                                     dflags, B.fn));
  Bins bn{B.bin_start, B.bx0, B.by0, B.nbx, B.nby, G->xf[0][0], G->xf[1][0]};
  // IB faces: about two per marker and component; the kernel strides over the list's length
  int nb = (int)std::min<long long>(148LL * 8, (4LL * B.nm + kT - 1) / kT + 1);
  FS_LAUNCH(G, "ib_gather", ib_gather_kernel<T><<<nb, kT, 0, G->stream>>>(
                                g, bn, B.X0, B.Y0, B.ds, B.fn, body_state, B.omega, B.centre[0], B.centre[1], B.iblist,
                                B.ibcount, (T*)B.num[0], (T*)B.den[0], (T*)B.num[1], (T*)B.den[1]));
}

template <typename T>
void ib_forces(fs_grid* G, double* body_state, double* advance, double dt) {
  IBDev& B = G->ib;
  const IBGeom g = make_geom(G);
  const int nlane = 2 * B.nm * 16;
  BodyODE ode{nullptr, B.mass, B.k, B.c, dt, B.active[0], B.active[1]};
  if (advance && B.mass > 0) ode.st = advance;
  FS_LAUNCH(G, "ib_force", force_kernel<T><<<(nlane + kT - 1) / kT, kT, 0, G->stream>>>(
                               g, B.nm, B.X0, B.Y0, B.ds, body_state, (const T*)B.f[0], (const T*)B.f[1], B.centre[0],
                               B.centre[1], G->rho, B.q, B.part, B.F, B.ticket, ode));
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
