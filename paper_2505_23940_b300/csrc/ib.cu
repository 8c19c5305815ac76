// Immersed-boundary and rigid-body kernels (§2.3.2-2.3.3 of the paper), 2-D bodies.
//
//   classify_solid   solid faces: crossing-number test of (face - w) against the
//                    rest polygon, every FP64 operation rounded on its own
//                    (__d*_rn) so the integer decision is the oracle's bit for bit;
//                    one block per face row finds the edges crossing the row's
//                    height once, then every face of the row counts the crossings
//                    to its right (both components in one launch)
//   classify_ib      IB faces: non-solid faces with a solid same-component neighbour
//   ib_target        F_N of Eq. (19) per marker and component (support nodes that are
//                    not solid) and the normalised scatter of Eq. (18): numerator and
//                    denominator of u_IB on IB faces; 16 lanes per (marker, component),
//                    one support node each, F_N summed by shuffles, one atomicAdd per
//                    IB node
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

struct Poly {
  const double* X;
  const double* Y;
  int n;
  double bb[4];
};

__device__ __forceinline__ bool inside_polygon(const Poly& P, double px, double py) {
  if (px < P.bb[0] || px > P.bb[1] || py < P.bb[2] || py > P.bb[3]) return false;
  bool in = false;
  for (int e = 0; e < P.n; ++e) {
    const double ax = P.X[e], ay = P.Y[e];
    const int f = (e + 1 == P.n) ? 0 : e + 1;
    const double bx = P.X[f], by = P.Y[f];
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
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  // x where each edge crosses the row's height (the order of the crossings does not matter to the parity)
  for (int e = threadIdx.x; e < P.n; e += blockDim.x) {
    const double ax = P.X[e], ay = P.Y[e];
    const int f = (e + 1 == P.n) ? 0 : e + 1;
    const double bx = P.X[f], by = P.Y[f];
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

// grid (blocks, 2 components)
__global__ void classify_ib_kernel(Flags F, int ex0, int ey0, int ex1, int ey1, int perx, int pery) {
  const int c = blockIdx.y;
  const int ex = c ? ex1 : ex0, ey = c ? ey1 : ey0;
  uint8_t* __restrict__ flags = c ? F.p[1] : F.p[0];
  const long long total = (long long)ex * ey;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % ex), j = (int)(t / ex);
    const uint8_t me = flags[t];
    if (me & 1) continue;
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

// F_N_i of Eq. (19) and the scatter of Eq. (18) in one pass: the 16 lanes of a
// (marker, component) pair evaluate delta_h at their support node once, sum
// F_N over the non-solid nodes by shuffles (every lane receives the sum), and
// the lanes whose node is an IB face add w = delta dV_i / F_N_i and w times the
// marker velocity to the numerator and denominator of u_IB.
template <typename T>
__global__ void ib_target_kernel(const IBGeom G, int nm, const double* __restrict__ X0, const double* __restrict__ Y0,
                                 const double* __restrict__ ds, const double* __restrict__ body, double omega,
                                 double cx, double cy, const Flags flags, double* __restrict__ fn, T* num0, T* den0,
                                 T* num1, T* den1) {
  const Lane L = lane_of(G, nm);
  double s = 0.0;
  T d = T(0);
  long long face = -1;
  double X = 0.0, Y = 0.0;
  if (L.live && L.b < G.width) {
    const int c = L.c;
    X = X0[L.m] + body[0];
    Y = Y0[L.m] + body[1];
    const int i = first_node(G, X, G.x0c[c], G.hx) + L.a, j = first_node(G, Y, G.y0c[c], G.hy) + L.b;
    if (i >= 0 && i < G.ex[c] && j >= 0 && j < G.ey[c]) {
      const size_t f = (size_t)j * G.ex[c] + i;
      const uint8_t fl = (c ? flags.p[1] : flags.p[0])[f];
      const T py = phi_kernel<T>(G.kind, T((node_y(G, c, j) - Y) * G.ihy));
      const T px = phi_kernel<T>(G.kind, T((node_x(G, c, i) - X) * G.ihx));
      d = px * py;
      if (!(fl & 1)) s = (double)d * G.ihxy;   // solid nodes are excluded from F_N
      if (fl & 2) face = (long long)f;
    }
  }
  const double F = sum16(s);
  if (L.live && (threadIdx.x & 15) == 0) fn[L.pair] = F;
  if (face >= 0 && F > 0.0) {
    const int c = L.c;
    const T w = T((double)d * G.ihxy * (ds[L.m] * G.hx) / F);
    // marker velocity: body translation plus surface rotation
    const double vm = c == 0 ? body[2] - omega * (Y - (cy + body[1])) : body[3] + omega * (X - (cx + body[0]));
    atomicAdd(c ? &num1[face] : &num0[face], w * T(vm));
    atomicAdd(c ? &den1[face] : &den0[face], w);
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
// component; then F = rho sum_i q_i dV_i and the torque rho sum_i dV_i (r_i x q_i)
// by the block that finishes last (the other blocks publish their q before
// taking a ticket; no block waits), in a fixed summation order, and, when asked,
// the body ODE step with that force.
template <typename T>
__global__ void __launch_bounds__(kT) force_kernel(const IBGeom G, int nm, const double* __restrict__ X0,
                                                   const double* __restrict__ Y0, const double* __restrict__ ds,
                                                   const double* body, const T* __restrict__ f0,
                                                   const T* __restrict__ f1, double cx, double cy, double rho,
                                                   double* __restrict__ q, double* __restrict__ F,
                                                   unsigned* __restrict__ ticket, const BodyODE ode) {
  const Lane L = lane_of(G, nm);
  double s = 0.0;
  if (L.live && L.b < G.width) {
    const int c = L.c;
    const T* f = c == 0 ? f0 : f1;
    const double X = X0[L.m] + body[0], Y = Y0[L.m] + body[1];
    const int i = first_node(G, X, G.x0c[c], G.hx) + L.a, j = first_node(G, Y, G.y0c[c], G.hy) + L.b;
    if (i >= 0 && i < G.ex[c] && j >= 0 && j < G.ey[c]) {
      const T py = phi_kernel<T>(G.kind, T((node_y(G, c, j) - Y) * G.ihy));
      const T px = phi_kernel<T>(G.kind, T((node_x(G, c, i) - X) * G.ihx));
      const double dvy = c == 0 ? G.hyv[j] : G.hfyv[j];
      s = (double)f[(size_t)j * G.ex[c] + i] * ((double)(px * py) * G.ihxy) * (G.hfx * dvy);
    }
  }
  s = sum16(s);
  if (L.live && (threadIdx.x & 15) == 0) q[L.pair] = -s;
  // the last block to finish reduces
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double s0[kT], s1[kT], s2[kT];
  const double bx = body[0], by = body[1];
  double a = 0, b = 0, tq = 0;
  for (int m = threadIdx.x; m < nm; m += blockDim.x) {
    const double dV = ds[m] * G.hx;
    const double qx = __ldcg(q + 2 * m), qy = __ldcg(q + 2 * m + 1);
    a += qx * dV;
    b += qy * dV;
    const double rx = X0[m] + bx - (cx + bx), ry = Y0[m] + by - (cy + by);
    tq += dV * (rx * qy - ry * qx);
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
  P.X = B.PX;
  P.Y = B.PY;
  P.n = B.nm;
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
  {
    const long long n = (long long)std::max(ex[0] * ey[0], ex[1] * ey[1]);
    int nb = (int)((n + kT - 1) / kT);
    if (nb > 148 * 8) nb = 148 * 8;
    FS_LAUNCH(G, "classify_ib", classify_ib_kernel<<<dim3(nb, 2), kT, 0, G->stream>>>(dflags, ex[0], ey[0], ex[1], ey[1],
                                                                                        G->per[0], G->per[1]));
  }
  const IBGeom g = make_geom(G);
  const int nlane = 2 * B.nm * 16;
  FS_LAUNCH(G, "ib_target", ib_target_kernel<T><<<(nlane + kT - 1) / kT, kT, 0, G->stream>>>(
                                g, B.nm, B.X0, B.Y0, B.ds, body_state, B.omega, B.centre[0], B.centre[1], dflags, B.fn,
                                (T*)B.num[0], (T*)B.den[0], (T*)B.num[1], (T*)B.den[1]));
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
                               B.centre[1], G->rho, B.q, B.F, B.ticket, ode));
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
