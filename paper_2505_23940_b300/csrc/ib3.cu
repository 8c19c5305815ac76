// Static 3-D immersed bodies made of axis-aligned boxes (fs_set_ib_boxes).
//
// The paper forces fixed 3-D bodies (cube roughness on a channel wall,
// obstacles; §3.4) with the direct forcing of §2.3.3: epsilon = 1 on solid
// faces (inside the body) and IB faces (fluid faces with a solid neighbour),
// where the target velocity of a body at rest is zero (Eqs. 5, 18, 23), and the
// hydrodynamic force is gathered at Lagrangian surface markers, Eq. (20):
//   q_i = -sum_faces f(x) delta_h(x - X_i) dv,   F = rho sum_i q_i dV_i.
// The body does not move, so the face classification is done once, when the
// body is set: a kernel per box marks the faces strictly inside it (work in
// proportion to the solid faces, whatever the number of boxes), a second pass
// marks the IB faces.  The forced velocity itself is applied inside the
// predictor kernels (stencil.cu); the force gather runs once per step with one
// thread per marker and component over the separable kernel support.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fs_internal.cuh"

namespace fs {

namespace {

// Face coordinate of index i along direction d for component c (the MAC face
// positions: face i of its own direction, cell centre i across).
__device__ __forceinline__ double face_pos(const double* xf, int i, bool own) {
  return own ? xf[i] : 0.5 * (xf[i] + xf[i + 1]);
}

struct BoxArgs {
  const double* boxes;
  const double* xf[3];
  int ext[3];
  uint8_t* flags;
  int c;
  double h[3], x0[3];
};

// One block per box: mark the faces of component c strictly inside it.
__global__ void mark_solid_kernel(const BoxArgs A) {
  const double* b = A.boxes + 6 * blockIdx.x;
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    // candidate index range, one face wider than needed on each side; the exact
    // test below decides
    const double off = d == A.c ? 0.0 : 0.5;
    lo[d] = max(0, (int)floor((b[2 * d] - A.x0[d]) / A.h[d] - off) - 1);
    hi[d] = min(A.ext[d] - 1, (int)ceil((b[2 * d + 1] - A.x0[d]) / A.h[d] - off) + 1);
  }
  const int nx = hi[0] - lo[0] + 1, ny = hi[1] - lo[1] + 1, nz = hi[2] - lo[2] + 1;
  if (nx <= 0 || ny <= 0 || nz <= 0) return;
  const long long tot = (long long)nx * ny * nz;
  for (long long t = threadIdx.x; t < tot; t += blockDim.x) {
    const int i = lo[0] + (int)(t % nx), j = lo[1] + (int)((t / nx) % ny), k = lo[2] + (int)(t / ((long long)nx * ny));
    const double x = face_pos(A.xf[0], i, A.c == 0), y = face_pos(A.xf[1], j, A.c == 1),
                 z = face_pos(A.xf[2], k, A.c == 2);
    if (x > b[0] && x < b[1] && y > b[2] && y < b[3] && z > b[4] && z < b[5])
      A.flags[i + (size_t)A.ext[0] * (j + (size_t)A.ext[1] * k)] = 1;
  }
}

// IB faces: not solid, with a solid same-component neighbour in any direction.
__global__ void mark_ib_kernel(uint8_t* flags, int ex, int ey, int ez, int px, int py, int pz) {
  const size_t n = (size_t)ex * ey * ez;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    if (flags[t] & 1) continue;
    const int i = (int)(t % ex), j = (int)((t / ex) % ey), k = (int)(t / ((size_t)ex * ey));
    const int e[3] = {ex, ey, ez}, p[3] = {i, j, k}, per[3] = {px, py, pz};
    bool nb = false;
    for (int d = 0; d < 3 && !nb; ++d)
      for (int s = -1; s <= 1 && !nb; s += 2) {
        int q[3] = {i, j, k};
        q[d] = p[d] + s;
        if (q[d] < 0 || q[d] >= e[d]) {
          if (!per[d]) continue;
          q[d] = (q[d] + e[d]) % e[d];
        }
        nb = flags[q[0] + (size_t)ex * (q[1] + (size_t)ey * q[2])] & 1;
      }
    if (nb) flags[t] = 2;
  }
}

// phi of Eq. (22) (Peskin 4-point) or the 3-point kernel of Roma, Peskin & Berger,
// in the field precision (FP32 IB transfers in mixed mode)
template <typename T>
__device__ __forceinline__ T phi3(int kind, T r) {
  const T a = fabs(r);
  if (kind == FS_PESKIN4) {
    if (a <= T(1)) return (T(3) - T(2) * a + sqrt(fmax(T(1) + T(4) * a - T(4) * a * a, T(0)))) / T(8);
    if (a <= T(2)) return (T(5) - T(2) * a - sqrt(fmax(T(-7) + T(12) * a - T(4) * a * a, T(0)))) / T(8);
    return T(0);
  }
  if (a <= T(0.5)) return (T(1) + sqrt(fmax(T(1) - T(3) * a * a, T(0)))) / T(3);
  if (a <= T(1.5)) {
    const T b = T(1) - a;
    return (T(5) - T(3) * a - sqrt(fmax(T(1) - T(3) * b * b, T(0)))) / T(6);
  }
  return T(0);
}

struct GatherArgs {
  int nm, kind, w;           // markers, kernel, support width
  const int* gi;             // SoA 3 * nm: marker cell index per direction, floor((X - x0) / h)
  const void* gf;            // SoA 3 * nm: its fraction in the cell, in the field precision
  const double* dV;
  double h[3];               // uniform spacing
  int ext[3][3];             // extents per component
  int per[3];
  double dv, rho;
  double* q;                 // SoA 3 * nm
  double* part;              // per-block sums of F (3 per block)
  unsigned* ticket;          // blocks finished (reset by the last one)
  double* F;
};

// One thread per marker: the separable weights of the two face families of
// every direction (a component's own faces, offset 0, and the faces across,
// offset 1/2) are formed once and serve the three components.  The marker's
// position in grid units comes as a cell index and a fraction (computed in FP64
// once, when the body is attached: the body is static), so the weights take no
// FP64 arithmetic; the support sums run in the field precision, q and the body
// force in FP64.  F is summed per block in a fixed tree and the block that
// finishes last adds the block sums in a fixed order (no block waits): the
// force is bitwise reproducible.
template <typename T, int W>
__global__ void __launch_bounds__(256) gather_kernel(const GatherArgs A, const T* __restrict__ f0,
                                                     const T* __restrict__ f1, const T* __restrict__ f2) {
  __shared__ double red[3][8];
  __shared__ bool last;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  double contrib[3] = {0.0, 0.0, 0.0};
  if (m < A.nm) {
    const T* gf = static_cast<const T*>(A.gf);
    int base[3][2];
    T wgt[3][2][W];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int gi = A.gi[d * A.nm + m];
      const T fr = gf[d * A.nm + m];
      const T ih = T(1.0 / A.h[d]);
#pragma unroll
      for (int fam = 0; fam < 2; ++fam) {
        // position s = gi + fr - off in units of this family's nodes (off = 1/2 across the component)
        T t = fr - (fam ? T(0.5) : T(0));
        const T k = floor(t);
        const int si = gi + (int)k;
        t -= k;                                    // in [0, 1)
        // faces within the support |s - i| < W / 2
        const int b0 = W == 4 ? si - 1 : si + (int)floor(t + T(0.5)) - 1;
        base[d][fam] = b0;
#pragma unroll
        for (int a = 0; a < W; ++a) wgt[d][fam][a] = phi3<T>(A.kind, T(si - (b0 + a)) + t) * ih;
      }
    }
    const T* fs[3] = {f0, f1, f2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T* f = fs[c];
      const int* e = A.ext[c];
      const int fx = c == 0 ? 0 : 1, fy = c == 1 ? 0 : 1, fz = c == 2 ? 0 : 1;
      T sum = T(0);
#pragma unroll
      for (int cz = 0; cz < W; ++cz) {
        int k = base[2][fz] + cz;
        if (k < 0 || k >= e[2]) {
          if (!A.per[2]) continue;
          k = (k % e[2] + e[2]) % e[2];
        }
#pragma unroll
        for (int cy = 0; cy < W; ++cy) {
          int j = base[1][fy] + cy;
          if (j < 0 || j >= e[1]) {
            if (!A.per[1]) continue;
            j = (j % e[1] + e[1]) % e[1];
          }
          const T wyz = wgt[2][fz][cz] * wgt[1][fy][cy];
          const T* row = f + (size_t)e[0] * (j + (size_t)e[1] * k);
          T rs = T(0);
#pragma unroll
          for (int cx = 0; cx < W; ++cx) {
            int i = base[0][fx] + cx;
            if (i < 0 || i >= e[0]) {
              if (!A.per[0]) continue;
              i = (i % e[0] + e[0]) % e[0];
            }
            rs += __ldg(row + i) * wgt[0][fx][cx];
          }
          sum += rs * wyz;
        }
      }
      const double qv = -(double)sum * A.dv;
      A.q[c * A.nm + m] = qv;
      contrib[c] = A.rho * qv * A.dV[m];
    }
  }
  for (int cc = 0; cc < 3; ++cc)
    for (int o = 16; o > 0; o >>= 1) contrib[cc] += __shfl_down_sync(0xffffffffu, contrib[cc], o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0)
    for (int cc = 0; cc < 3; ++cc) red[cc][w] = contrib[cc];
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) v += red[threadIdx.x][q];
    A.part[3 * blockIdx.x + threadIdx.x] = v;
  }
  // the last block to finish adds the block sums in block order
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(A.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
    for (int cc = 0; cc < 3; ++cc) v[cc] += __ldcg(A.part + 3 * b + cc);
  for (int cc = 0; cc < 3; ++cc)
    for (int o = 16; o > 0; o >>= 1) v[cc] += __shfl_down_sync(0xffffffffu, v[cc], o);
  __syncthreads();
  if (l == 0)
    for (int cc = 0; cc < 3; ++cc) red[cc][w] = v[cc];
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += red[threadIdx.x][q];
    A.F[threadIdx.x] = t;
  }
  if (threadIdx.x == 0) *A.ticket = 0u;
}

}  // namespace

void free_ib3(fs_grid* G) {
  IB3Dev& B = G->ib3;
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  F(B.boxes);
  F(B.X);
  F(B.dV);
  for (int c = 0; c < 3; ++c) {
    F(B.flags[c]);
    F(B.f[c]);
  }
  F(B.q);
  F(B.F);
  F(B.gi);
  F(B.gf);
  F(B.part);
  F(B.ticket);
  B = IB3Dev();
  G->has_ib3 = false;
}

template <typename T>
void ib3_forces(fs_grid* G) {
  IB3Dev& B = G->ib3;
  if (B.nm == 0) return;
  GatherArgs A;
  A.nm = B.nm;
  A.kind = B.kernel;
  A.w = B.kernel == FS_PESKIN4 ? 4 : 3;
  A.gi = B.gi;
  A.gf = B.gf;
  A.dV = B.dV;
  const int n[3] = {G->nx, G->ny, G->nz};
  for (int d = 0; d < 3; ++d) {
    A.h[d] = G->h[d][0];
    A.per[d] = G->per[d];
    for (int c = 0; c < 3; ++c) A.ext[c][d] = n[d] + ((c == d && !G->per[d]) ? 1 : 0);
  }
  A.dv = A.h[0] * A.h[1] * A.h[2];
  A.rho = G->rho;
  A.q = B.q;
  A.F = B.F;
  A.part = B.part;
  A.ticket = B.ticket;
  const int nb = (B.nm + 255) / 256;
  if (A.w == 4)
    FS_LAUNCH(G, "ib3_force_gather", gather_kernel<T, 4><<<nb, 256, 0, G->stream>>>(
                                         A, (const T*)B.f[0], (const T*)B.f[1], (const T*)B.f[2]));
  else
    FS_LAUNCH(G, "ib3_force_gather", gather_kernel<T, 3><<<nb, 256, 0, G->stream>>>(
                                         A, (const T*)B.f[0], (const T*)B.f[1], (const T*)B.f[2]));
  B.have_forces = true;
}

template void ib3_forces<float>(fs_grid*);
template void ib3_forces<double>(fs_grid*);

}  // namespace fs

using namespace fs;

namespace {
bool uniform_h(const std::vector<double>& h) {
  for (double v : h)
    if (std::fabs(v - h[0]) > 1e-12 * std::fabs(h[0])) return false;
  return true;
}

template <typename T>
cudaError_t upload_vec(T** p, const std::vector<T>& v) {
  cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(v.size(), 1) * sizeof(T));
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}
}  // namespace

extern "C" int fs_set_ib_boxes(fs_grid* G, int nbox, const double* boxes, int nm, const double* X, const double* dV,
                               int delta_kernel) {
  if (!G) return set_error(FS_ERR_ARG, "NULL grid");
  if (G->dim != 3) return set_error(FS_ERR_UNSUPPORTED, "box bodies are provided for 3-D grids");
  if (G->scheme != FS_FE) return set_error(FS_ERR_UNSUPPORTED, "immersed bodies use forward Euler");
  if (nbox < 0 || nm < 0 || (nbox > 0 && !boxes) || (nm > 0 && (!X || !dV)))
    return set_error(FS_ERR_ARG, "fs_set_ib_boxes: bad counts or NULL arrays");
  if (delta_kernel != FS_PESKIN4 && delta_kernel != FS_ROMA3) return set_error(FS_ERR_ARG, "unknown delta kernel");
  for (int d = 0; d < 3; ++d)
    if (!uniform_h(G->h[d])) return set_error(FS_ERR_ARG, "box bodies need uniform spacing in x, y and z");
  for (int b = 0; b < nbox; ++b)
    for (int d = 0; d < 3; ++d)
      if (!(boxes[6 * b + 2 * d] < boxes[6 * b + 2 * d + 1])) return set_error(FS_ERR_ARG, "box with lo >= hi");
  free_ib3(G);
  IB3Dev& B = G->ib3;
  B.nbox = nbox;
  B.nm = nm;
  B.kernel = delta_kernel;
  std::vector<double> bx(boxes, boxes + 6 * (size_t)nbox), xs(3 * (size_t)nm), dv(dV, dV + nm);
  for (int m = 0; m < nm; ++m)
    for (int d = 0; d < 3; ++d) xs[(size_t)d * nm + m] = X[3 * (size_t)m + d];
  // marker positions in grid units: cell index and fraction per direction (FP64 here, once)
  std::vector<int> gi(3 * (size_t)nm);
  std::vector<double> gfr(3 * (size_t)nm);
  for (int d = 0; d < 3; ++d)
    for (int m = 0; m < nm; ++m) {
      const double g = (xs[(size_t)d * nm + m] - G->xf[d][0]) / G->h[d][0];
      const double fl = std::floor(g);
      gi[(size_t)d * nm + m] = (int)fl;
      gfr[(size_t)d * nm + m] = g - fl;
    }
  const int nblk = std::max(1, (nm + 255) / 256);
  bool ok = upload_vec(&B.boxes, bx) == cudaSuccess && upload_vec(&B.X, xs) == cudaSuccess &&
            upload_vec(&B.dV, dv) == cudaSuccess && cudaMalloc(&B.q, std::max(3 * nm, 1) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&B.F, 3 * sizeof(double)) == cudaSuccess && upload_vec(&B.gi, gi) == cudaSuccess &&
            cudaMalloc(&B.part, 3 * (size_t)nblk * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&B.ticket, sizeof(unsigned)) == cudaSuccess &&
            cudaMemset(B.ticket, 0, sizeof(unsigned)) == cudaSuccess;
  if (ok && G->prec == FS_MIXED) {
    std::vector<float> g32(gfr.begin(), gfr.end());
    float* p = nullptr;
    ok = upload_vec(&p, g32) == cudaSuccess;
    B.gf = p;
  } else if (ok) {
    double* p = nullptr;
    ok = upload_vec(&p, gfr) == cudaSuccess;
    B.gf = p;
  }
  const size_t es = G->prec == FS_MIXED ? sizeof(float) : sizeof(double);
  const int n[3] = {G->nx, G->ny, G->nz};
  for (int c = 0; c < 3 && ok; ++c) {
    int ext[3];
    size_t cnt = 1;
    for (int d = 0; d < 3; ++d) {
      ext[d] = n[d] + ((c == d && !G->per[d]) ? 1 : 0);
      cnt *= ext[d];
    }
    ok = cudaMalloc(&B.flags[c], cnt) == cudaSuccess && cudaMalloc(&B.f[c], cnt * es) == cudaSuccess &&
         cudaMemsetAsync(B.flags[c], 0, cnt, G->stream) == cudaSuccess &&
         cudaMemsetAsync(B.f[c], 0, cnt * es, G->stream) == cudaSuccess;
    if (!ok) break;
    BoxArgs A;
    A.boxes = B.boxes;
    for (int d = 0; d < 3; ++d) {
      A.xf[d] = G->xf64[d];
      A.ext[d] = ext[d];
      A.h[d] = G->h[d][0];
      A.x0[d] = G->xf[d][0];
    }
    A.flags = B.flags[c];
    A.c = c;
    if (nbox > 0) FS_LAUNCH(G, "ib3_classify", mark_solid_kernel<<<nbox, 256, 0, G->stream>>>(A));
    const int blocks = (int)std::min<size_t>((cnt + 255) / 256, 148 * 16);
    FS_LAUNCH(G, "ib3_classify", mark_ib_kernel<<<blocks, 256, 0, G->stream>>>(B.flags[c], ext[0], ext[1], ext[2],
                                                                                G->per[0], G->per[1], G->per[2]));
  }
  if (ok) ok = cudaMemsetAsync(B.F, 0, 3 * sizeof(double), G->stream) == cudaSuccess;
  if (!ok) {
    free_ib3(G);
    return set_error(FS_ERR_CUDA, "allocating the box body");
  }
  G->has_ib3 = true;
  return cuda_check(cudaGetLastError(), "fs_set_ib_boxes");
}
