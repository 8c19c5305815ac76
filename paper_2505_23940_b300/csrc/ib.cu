// Immersed-boundary and rigid-body kernels (§2.3.2-2.3.3 of the paper), 2-D bodies.
//
//   classify_solid   solid faces: crossing-number test of (face - w) against the
//                    rest polygon, every FP64 operation rounded on its own
//                    (__d*_rn) so the integer decision is the oracle's bit for bit
//   classify_ib      IB faces: non-solid faces with a solid same-component neighbour
//   fn_gather        F_N of Eq. (19) per marker and component (support nodes that are not solid)
//   ib_scatter       Eq. (18), normalised: numerator / denominator of u_IB on IB faces;
//                    markers are sorted by cell, contributions to the same face are
//                    summed inside the warp (match_any + shuffles) before one atomicAdd
//   force_gather     q_i of Eq. (20) per marker (FP64 sums)
//   force_reduce     F = rho sum q_i dV_i and torque, one CTA, fixed order (FP64)
//   rk4              Eq. (12), classical RK4 with the force frozen (one thread, FP64)
//
// Kernel evaluation: node offsets from markers are formed in FP64, the
// kernel phi in the field precision T.
#include <cuda_runtime.h>

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

__global__ void classify_solid_kernel(uint8_t* __restrict__ flags, int c, int ex, int ey, const double* xf,
                                      const double* yf, const double* body, Poly P) {
  const long long total = (long long)ex * ey;
  const double wx = body[0], wy = body[1];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % ex), j = (int)(t / ex);
    double px, py;
    face_pos(c, i, j, xf, yf, px, py);
    flags[t] = inside_polygon(P, __dsub_rn(px, wx), __dsub_rn(py, wy)) ? 1 : 0;
  }
}

__global__ void classify_ib_kernel(uint8_t* __restrict__ flags, int ex, int ey, int perx, int pery) {
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

struct Flags {
  uint8_t* p[2];
};

struct IBGeom {
  int ex[2], ey[2];
  double x0c[2], y0c[2];   // position of node (0, 0) of each component
  double hx, hy;
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

// F_N_i for both components (Eq. 19)
template <typename T>
__global__ void fn_gather_kernel(const IBGeom G, int nm, const double* __restrict__ X0, const double* __restrict__ Y0,
                                 const double* __restrict__ body, const Flags flags, double* __restrict__ fn) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nm) return;
  const int m = t >> 1, c = t & 1;
  const double X = X0[m] + body[0], Y = Y0[m] + body[1];
  const int i0 = first_node(G, X, G.x0c[c], G.hx), j0 = first_node(G, Y, G.y0c[c], G.hy);
  double s = 0.0;
  for (int b = 0; b < G.width; ++b) {
    const int j = j0 + b;
    if (j < 0 || j >= G.ey[c]) continue;
    const T py = T(phi_kernel<T>(G.kind, T((node_y(G, c, j) - Y) / G.hy)));
    for (int a = 0; a < G.width; ++a) {
      const int i = i0 + a;
      if (i < 0 || i >= G.ex[c]) continue;
      if (flags.p[c][(size_t)j * G.ex[c] + i] & 1) continue;   // solid nodes excluded
      const T px = phi_kernel<T>(G.kind, T((node_x(G, c, i) - X) / G.hx));
      s += (double)(px * py) / (G.hx * G.hy);
    }
  }
  fn[t] = s;
}

// Eq. (18): num += w_i wdot_i, den += w_i on IB faces, w_i = delta dV_i / F_N_i.
template <typename T>
__global__ void ib_scatter_kernel(const IBGeom G, int nm, const double* __restrict__ X0, const double* __restrict__ Y0,
                                  const double* __restrict__ ds, const double* __restrict__ body, double omega,
                                  double cx, double cy, const Flags flags, const double* __restrict__ fn,
                                  T* num0, T* den0, T* num1, T* den1) {
  const int nn = G.width * G.width;
  const long long total = 2ll * nm * nn;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long key = -1;
  T wv = T(0), w = T(0);
  int c = 0;
  if (t < total) {
    // thread order: component, node, marker (consecutive lanes = consecutive sorted markers)
    c = (int)(t / ((long long)nm * nn));
    const int r = (int)(t - (long long)c * nm * nn);
    const int node = r / nm, m = r - node * nm;
    const int a = node % G.width, b = node / G.width;
    const double X = X0[m] + body[0], Y = Y0[m] + body[1];
    const int i = first_node(G, X, G.x0c[c], G.hx) + a, j = first_node(G, Y, G.y0c[c], G.hy) + b;
    if (i >= 0 && i < G.ex[c] && j >= 0 && j < G.ey[c]) {
      const size_t f = (size_t)j * G.ex[c] + i;
      if (flags.p[c][f] & 2) {
        const double F = fn[2 * m + c];
        if (F > 0.0) {
          const T d = phi_kernel<T>(G.kind, T((node_x(G, c, i) - X) / G.hx)) *
                      phi_kernel<T>(G.kind, T((node_y(G, c, j) - Y) / G.hy));
          w = T((double)d / (G.hx * G.hy) * (ds[m] * G.hx) / F);
          // marker velocity: body translation plus surface rotation
          const double vm = c == 0 ? body[2] - omega * (Y - (cy + body[1])) : body[3] + omega * (X - (cx + body[0]));
          wv = w * T(vm);
          key = (long long)c << 40 | (long long)f;
        }
      }
    }
  }
  // warp-level reduction of contributions that hit the same face, then one atomic per face
  const unsigned full = 0xffffffffu;
  const unsigned grp = __match_any_sync(full, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(grp) - 1;
  T sw = T(0), swv = T(0);
  for (int src = 0; src < 32; ++src) {
    const T a = __shfl_sync(full, w, src), b = __shfl_sync(full, wv, src);
    if ((grp >> src) & 1u) {
      sw += a;
      swv += b;
    }
  }
  if (key >= 0 && lane == leader) {
    const size_t f = (size_t)(key & ((1ll << 40) - 1));
    if ((key >> 40) == 0) {
      atomicAdd(&num0[f], swv);
      atomicAdd(&den0[f], sw);
    } else {
      atomicAdd(&num1[f], swv);
      atomicAdd(&den1[f], sw);
    }
  }
}

// q_i = - sum_x f(x) delta_h(x - X_i) dv(x)   (Eq. 20), per marker and component
template <typename T>
__global__ void force_gather_kernel(const IBGeom G, int nm, const double* __restrict__ X0,
                                    const double* __restrict__ Y0, const double* __restrict__ body,
                                    const T* __restrict__ f0, const T* __restrict__ f1, double* __restrict__ q) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nm) return;
  const int m = t >> 1, c = t & 1;
  const T* f = c == 0 ? f0 : f1;
  const double X = X0[m] + body[0], Y = Y0[m] + body[1];
  const int i0 = first_node(G, X, G.x0c[c], G.hx), j0 = first_node(G, Y, G.y0c[c], G.hy);
  double s = 0.0;
  for (int b = 0; b < G.width; ++b) {
    const int j = j0 + b;
    if (j < 0 || j >= G.ey[c]) continue;
    const T py = phi_kernel<T>(G.kind, T((node_y(G, c, j) - Y) / G.hy));
    const double dvy = c == 0 ? G.hyv[j] : G.hfyv[j];
    for (int a = 0; a < G.width; ++a) {
      const int i = i0 + a;
      if (i < 0 || i >= G.ex[c]) continue;
      const T px = phi_kernel<T>(G.kind, T((node_x(G, c, i) - X) / G.hx));
      const double d = (double)(px * py) / (G.hx * G.hy);
      s += (double)f[(size_t)j * G.ex[c] + i] * d * (G.hfx * dvy);
    }
  }
  q[t] = -s;
}

// F = rho sum_i q_i dV_i, torque = rho sum_i dV_i (r_i x q_i); one CTA, fixed summation order.
__global__ void force_reduce_kernel(int nm, const double* __restrict__ X0, const double* __restrict__ Y0,
                                    const double* __restrict__ ds, const double* __restrict__ body, double cx,
                                    double cy, double hx, double rho, const double* __restrict__ q,
                                    double* __restrict__ F) {
  __shared__ double s0[kT], s1[kT], s2[kT];
  double a = 0, b = 0, tq = 0;
  for (int m = threadIdx.x; m < nm; m += blockDim.x) {
    const double dV = ds[m] * hx;
    const double qx = q[2 * m], qy = q[2 * m + 1];
    a += qx * dV;
    b += qy * dV;
    const double rx = X0[m] + body[0] - (cx + body[0]), ry = Y0[m] + body[1] - (cy + body[1]);
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
  }
}

// Eq. (12) with F frozen over the step: classical RK4 per active DOF.
__global__ void rk4_kernel(double* __restrict__ st, const double* __restrict__ F, double m, double k, double c,
                           int ax, int ay, double dt) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
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

IBGeom make_geom(const fs_grid* G) {
  IBGeom g;
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
  for (int c = 0; c < 2; ++c) {
    const int ex = G->nx + ((c == 0 && !G->per[0]) ? 1 : 0), ey = G->ny + ((c == 1 && !G->per[1]) ? 1 : 0);
    const long long n = (long long)ex * ey;
    int nb = (int)((n + kT - 1) / kT);
    if (nb > 148 * 16) nb = 148 * 16;
    FS_LAUNCH(G, "classify_solid", classify_solid_kernel<<<nb, kT, 0, G->stream>>>(B.flags[c], c, ex, ey, G->xf64[0], G->xf64[1], body_state, P));
  }
  for (int c = 0; c < 2; ++c) {
    const int ex = G->nx + ((c == 0 && !G->per[0]) ? 1 : 0), ey = G->ny + ((c == 1 && !G->per[1]) ? 1 : 0);
    const long long n = (long long)ex * ey;
    int nb = (int)((n + kT - 1) / kT);
    if (nb > 148 * 16) nb = 148 * 16;
    FS_LAUNCH(G, "classify_ib", classify_ib_kernel<<<nb, kT, 0, G->stream>>>(B.flags[c], ex, ey, G->per[0], G->per[1]));
  }
  const IBGeom g = make_geom(G);
  Flags dflags;
  dflags.p[0] = B.flags[0];
  dflags.p[1] = B.flags[1];
  FS_LAUNCH(G, "fn_gather", fn_gather_kernel<T><<<(2 * B.nm + 127) / 128, 128, 0, G->stream>>>(g, B.nm, B.X0, B.Y0, body_state, dflags, B.fn));
  const long long total = 2ll * B.nm * g.width * g.width;
  FS_LAUNCH(G, "ib_scatter", ib_scatter_kernel<T><<<(int)((total + kT - 1) / kT), kT, 0, G->stream>>>(
      g, B.nm, B.X0, B.Y0, B.ds, body_state, B.omega, B.centre[0], B.centre[1], dflags, B.fn, (T*)B.num[0],
      (T*)B.den[0], (T*)B.num[1], (T*)B.den[1]));
}

template <typename T>
void ib_forces(fs_grid* G, const double* body_state) {
  IBDev& B = G->ib;
  const IBGeom g = make_geom(G);
  FS_LAUNCH(G, "force_gather", force_gather_kernel<T><<<(2 * B.nm + 127) / 128, 128, 0, G->stream>>>(g, B.nm, B.X0, B.Y0, body_state,
                                                                          (const T*)B.f[0], (const T*)B.f[1], B.q));
  FS_LAUNCH(G, "force_reduce", force_reduce_kernel<<<1, kT, 0, G->stream>>>(B.nm, B.X0, B.Y0, B.ds, body_state, B.centre[0], B.centre[1], G->hx,
                                               G->rho, B.q, B.F));
  B.have_forces = true;
}

void body_rk4(fs_grid* G, double* body_state, double dt) {
  IBDev& B = G->ib;
  if (B.mass <= 0) return;
  FS_LAUNCH(G, "rk4", rk4_kernel<<<1, 32, 0, G->stream>>>(body_state, B.F, B.mass, B.k, B.c, B.active[0], B.active[1], dt));
}

template void ib_prepare<float>(fs_grid*, const double*);
template void ib_prepare<double>(fs_grid*, const double*);
template void ib_forces<float>(fs_grid*, const double*);
template void ib_forces<double>(fs_grid*, const double*);

}  // namespace fs
