// Direct solve of the discrete pressure Poisson equation D G phi = b (Eq. 9 of
// the paper).  The paper iterates with CG; every Krylov iteration converges to
// the same unique zero-mean solution, which this solver computes directly:
//
//   x: real-to-complex DFT (periodic) or DCT-II (Neumann), two rows per complex
//      FFT, output "real-packed" so the spectrum has exactly the cell count
//        slot 0 = Re X_0, slot 1 = Re X_{n/2}, slots 2m, 2m+1 = Re, Im X_m
//   z: (3-D) complex FFT of slot pairs (2m, 2m+1) along z; the pair m = 0 holds
//      two real sequences and is split into two real-packed z spectra
//   y: wall-bounded (possibly stretched) y: per wavenumber, the remaining
//      tridiagonal system in FP64 (partitioned Thomas with factors precomputed
//      per eigenvalue; the singular zero mode pinned and shifted to zero mean).
//      Periodic y is uniform and its operator circulant: a complex DFT along y
//      of slot pairs, division by the eigenvalue sum, inverse DFT, all in one
//      kernel in the field precision; the zero mode is set to zero (zero mean).
//   inverse z, inverse x.
//
// FFTs: mixed-radix (2, 3, 4, 5, 7, 11, 13) Stockham autosort in shared memory,
// one complex line per group of butterflies, whole lines resident per CTA.
// Precision: the field type T for transforms (FP32 in mixed mode), FP64 for the
// tridiagonal elimination in both modes.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "fs_internal.cuh"
#include "fpconv.cuh"
#include "tma.cuh"

namespace fs {

template <typename T>
struct cplx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cplx<T> cconj(cplx<T> a) {
  return {a.x, -a.y};
}

struct Radices {
  int nst;
  int r[FS_MAX_RADIX_STAGES];
};

namespace {

constexpr int kMaxLines = 16;   // complex lines per FFT block (upper bound; the compile-time lengths use exactly this)

// One Stockham stage with compile-time radix R over `nlines` lines of length N.
// NC, NSC: compile-time line length and sub-transform size (0: the runtime values).
template <typename T, int R, int NC = 0, int NSC = 0>
__device__ __forceinline__ void stockham_stage(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int Nrt,
                                               int P, int nlines, int Nsrt, const cplx<T>* __restrict__ tw, bool inv) {
  const int N = NC ? NC : Nrt;
  const int Ns = NSC ? NSC : Nsrt;
  const int NR = N / R;
  const int nb = nlines * NR;
  const int tws = N / (Ns * R);
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    const int line = t / NR;
    const int jj = t - line * NR;
    const cplx<T>* a = in + line * P;
    cplx<T>* b = out + line * P;
    const int k = jj % Ns;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[r] = a[jj + r * NR];
      if (r > 0 && k > 0) {
        cplx<T> w = tw[r * k * tws];
        if (inv) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    // R-point DFT
    cplx<T> o[R];
    if (R == 2) {
      o[0] = {v[0].x + v[1].x, v[0].y + v[1].y};
      o[1] = {v[0].x - v[1].x, v[0].y - v[1].y};
    } else if (R == 4) {
      const cplx<T> s02 = {v[0].x + v[2].x, v[0].y + v[2].y}, d02 = {v[0].x - v[2].x, v[0].y - v[2].y};
      const cplx<T> s13 = {v[1].x + v[3].x, v[1].y + v[3].y}, d13 = {v[1].x - v[3].x, v[1].y - v[3].y};
      // -i * d13 (forward) or +i * d13 (inverse)
      const cplx<T> rot = inv ? cplx<T>{-d13.y, d13.x} : cplx<T>{d13.y, -d13.x};
      o[0] = {s02.x + s13.x, s02.y + s13.y};
      o[2] = {s02.x - s13.x, s02.y - s13.y};
      o[1] = {d02.x + rot.x, d02.y + rot.y};
      o[3] = {d02.x - rot.x, d02.y - rot.y};
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        cplx<T> s = v[0];
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cplx<T> w = tw[NR * ((q * r) % R)];
          if (inv) w.y = -w.y;
          const cplx<T> p = cmul(v[r], w);
          s.x += p.x;
          s.y += p.y;
        }
        o[q] = s;
      }
    }
    const int idxD = (jj / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) b[idxD + r * Ns] = o[r];
  }
}

// In-place (ping-pong) FFT of nlines lines of length N held in shared memory.
// Returns the buffer holding the result.
// BIG selects the instantiation that also carries radix 7, 11 and 13 stages;
// lengths with prime factors <= 5 use the one without, whose register count
// is not set by those large butterflies.
template <typename T, bool BIG>
__device__ cplx<T>* fft_smem(cplx<T>* a, cplx<T>* b, int N, int P, int nlines, const Radices& rad,
                             const cplx<T>* __restrict__ tw, bool inv) {
  int Ns = 1;
  for (int s = 0; s < rad.nst; ++s) {
    const int R = rad.r[s];
    switch (R) {
      case 2: stockham_stage<T, 2>(a, b, N, P, nlines, Ns, tw, inv); break;
      case 3: stockham_stage<T, 3>(a, b, N, P, nlines, Ns, tw, inv); break;
      case 4: stockham_stage<T, 4>(a, b, N, P, nlines, Ns, tw, inv); break;
      case 5: stockham_stage<T, 5>(a, b, N, P, nlines, Ns, tw, inv); break;
      default:
        if constexpr (BIG) {
          if (R == 7) stockham_stage<T, 7>(a, b, N, P, nlines, Ns, tw, inv);
          else if (R == 11) stockham_stage<T, 11>(a, b, N, P, nlines, Ns, tw, inv);
          else stockham_stage<T, 13>(a, b, N, P, nlines, Ns, tw, inv);
        }
        break;
    }
    __syncthreads();
    cplx<T>* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// Compile-time plans for the line lengths used most (64, 128, 192, 256): the
// radix sequence, stage sizes and every index division are constants.
constexpr int ct_radix(int n, int s) {
  int m = n, st = 0;
  while (m % 4 == 0 && m > 4) {
    if (st == s) return 4;
    m /= 4;
    ++st;
  }
  const int primes[7] = {4, 2, 3, 5, 7, 11, 13};
  for (int q = 0; q < 7; ++q)
    while (m % primes[q] == 0) {
      if (st == s) return primes[q];
      m /= primes[q];
      ++st;
    }
  return 1;
}

constexpr int ct_nstages(int n) {
  int st = 0;
  while (ct_radix(n, st) > 1) ++st;
  return st;
}

template <typename T, int N, int S, int NS>
__device__ __forceinline__ cplx<T>* fft_ct(cplx<T>* a, cplx<T>* b, int P, int nlines, const cplx<T>* __restrict__ tw,
                                          bool inv) {
  if constexpr (S >= ct_nstages(N)) {
    return a;
  } else {
    constexpr int R = ct_radix(N, S);
    stockham_stage<T, R, N, NS>(a, b, N, P, nlines, NS, tw, inv);
    __syncthreads();
    return fft_ct<T, N, S + 1, NS * R>(b, a, P, nlines, tw, inv);
  }
}

// PL: 0 generic plan with radices <= 5, 1 generic plan with radices up to 13,
// >= 2 the compile-time plan of length PL.
template <typename T, int PL>
__device__ __forceinline__ cplx<T>* fft_any(cplx<T>* a, cplx<T>* b, int N, int P, int nlines, const Radices& rad,
                                           const cplx<T>* __restrict__ tw, bool inv) {
  if constexpr (PL >= 2) return fft_ct<T, PL, 0, 1>(a, b, P, nlines, tw, inv);
  else return fft_smem<T, PL == 1>(a, b, N, P, nlines, rad, tw, inv);
}

// ---------------------------------------------------------------------------
// x transforms: rows of length N = nx, two rows per complex line.
// mode 0: periodic DFT (real-packed output), mode 1: DCT-II.
// DIV: the rows are not read from `data` but formed on the fly as the
// divergence D[(1 - eps) u* + eps u_c] of Eq. (9) (row r = j + ny k).
template <typename T, int PL, bool DIV>
__global__ void __launch_bounds__(256) xfwd_kernel(T* __restrict__ data, int Nrt, int rows, int lpb, int mode, Radices rad,
                            const cplx<T>* __restrict__ tw, const cplx<T>* __restrict__ dtw,
                            const DivArgs<T> dv) {
  extern __shared__ unsigned char smem_raw[];
  const int N = PL >= 2 ? PL : Nrt;
  cplx<T>* A = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* B = A + (size_t)lpb * N;
  const int line0 = blockIdx.x * lpb;
  const int nl = min(lpb, (rows + 1) / 2 - line0);
  // (j, k) of the block's rows, formed once (rows r = j + ny k)
  __shared__ int rowj[2 * kMaxLines], rowk[2 * kMaxLines];
  if constexpr (DIV) {
    if (threadIdx.x < 2 * nl) {
      const int r = 2 * line0 + threadIdx.x;
      rowk[threadIdx.x] = r / dv.g.ny;
      rowj[threadIdx.x] = r - rowk[threadIdx.x] * dv.g.ny;
    }
    __syncthreads();
  }
  bool done = false;
  if constexpr (DIV && PL >= 2 && PL % 4 == 0) {
    if (dv.vec4 && mode == 0) {
      // four cells per thread: row-vector loads of u*, v*, w*
      constexpr int NQ = PL / 4;
      for (int Q = threadIdx.x; Q < nl * NQ; Q += blockDim.x) {
        const int l = Q / NQ, i0 = 4 * (Q - l * NQ);
        const Vec4<T> da = div4_at(dv, i0, rowj[2 * l], rowk[2 * l]);
        Vec4<T> db = {{T(0), T(0), T(0), T(0)}};
        if (2 * (line0 + l) + 1 < rows) db = div4_at(dv, i0, rowj[2 * l + 1], rowk[2 * l + 1]);
#pragma unroll
        for (int e = 0; e < 4; ++e) A[l * N + i0 + e] = {da.v[e], db.v[e]};
      }
      done = true;
    }
  }
  // loads are batched (KB elements per thread in flight) before the shared-memory stores
  constexpr int KB = 4;
  for (int t0 = threadIdx.x; !done && t0 < nl * N; t0 += KB * blockDim.x) {
    T va[KB], vb[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int t = t0 + q * blockDim.x;
      va[q] = vb[q] = T(0);
      if (t < nl * N) {
        const int l = t / N, i = t - l * N;
        const int r0 = 2 * (line0 + l), r1 = r0 + 1;
        if constexpr (DIV) {
          va[q] = div_at(dv, i, rowj[2 * l], rowk[2 * l]);
          if (r1 < rows) vb[q] = div_at(dv, i, rowj[2 * l + 1], rowk[2 * l + 1]);
        } else {
          va[q] = data[(size_t)r0 * N + i];
          if (r1 < rows) vb[q] = data[(size_t)r1 * N + i];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int t = t0 + q * blockDim.x;
      if (t < nl * N) {
        const int l = t / N, i = t - l * N;
        int dst = i;
        if (mode == 1) dst = (i & 1) ? N - 1 - (i >> 1) : (i >> 1);   // even samples forward, odd reversed
        A[l * N + dst] = {va[q], vb[q]};
      }
    }
  }
  __syncthreads();
  cplx<T>* Z = fft_any<T, PL>(A, B, N, N, nl, rad, tw, false);
  for (int t = threadIdx.x; t < nl * N; t += blockDim.x) {
    const int l = t / N, s = t - l * N;
    const int r0 = 2 * (line0 + l), r1 = r0 + 1;
    int m;
    bool im = false;
    if (mode == 0) {
      m = s == 0 ? 0 : (s == 1 ? N / 2 : s >> 1);
      im = s >= 2 && (s & 1);
    } else {
      m = s;
    }
    const cplx<T> z = Z[l * N + m], zr = Z[l * N + (m == 0 ? 0 : N - m)];
    // spectra of the two real rows: XA = (Z + conj Zr) / 2, XB = (Z - conj Zr) / (2 i)
    const cplx<T> xa = {T(0.5) * (z.x + zr.x), T(0.5) * (z.y - zr.y)};
    const cplx<T> xb = {T(0.5) * (z.y + zr.y), T(0.5) * (zr.x - z.x)};
    T oa, ob;
    if (mode == 0) {
      oa = im ? xa.y : xa.x;
      ob = im ? xb.y : xb.x;
    } else {
      const cplx<T> w = dtw[m];   // exp(-i pi m / (2 N))
      oa = w.x * xa.x - w.y * xa.y;
      ob = w.x * xb.x - w.y * xb.y;
    }
    data[(size_t)r0 * N + s] = oa;
    if (r1 < rows) data[(size_t)r1 * N + s] = ob;
  }
}

template <typename T>
__device__ __forceinline__ cplx<T> unpack_packed(const T* __restrict__ row, int N, int k) {
  // Hermitian spectrum X[k] from a real-packed row
  if (k == 0) return {row[0], T(0)};
  if (2 * k == N) return {row[1], T(0)};
  if (2 * k < N) return {row[2 * k], row[2 * k + 1]};
  const int m = N - k;
  return {row[2 * m], -row[2 * m + 1]};
}

template <typename T, int PL>
__global__ void __launch_bounds__(256) xinv_kernel(T* __restrict__ data, int Nrt, int rows, int lpb, int mode, Radices rad,
                            const cplx<T>* __restrict__ tw, const cplx<T>* __restrict__ dtw) {
  extern __shared__ unsigned char smem_raw[];
  const int N = PL >= 2 ? PL : Nrt;
  cplx<T>* A = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* B = A + (size_t)lpb * N;
  const int line0 = blockIdx.x * lpb;
  const int nl = min(lpb, (rows + 1) / 2 - line0);
  constexpr int KB = 4;
  for (int t0 = threadIdx.x; t0 < nl * N; t0 += KB * blockDim.x) {
    cplx<T> z[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int t = t0 + q * blockDim.x;
      z[q] = {T(0), T(0)};
      if (t < nl * N) {
        const int l = t / N, k = t - l * N;
        const int r0 = 2 * (line0 + l), r1 = r0 + 1;
        const T* ra = data + (size_t)r0 * N;
        const T* rb = data + (size_t)r1 * N;
        cplx<T> xa, xb;
        if (mode == 0) {
          xa = unpack_packed(ra, N, k);
          xb = r1 < rows ? unpack_packed(rb, N, k) : cplx<T>{T(0), T(0)};
        } else {
          // V[k] = exp(i pi k / 2N) (X[k] - i X[N-k]), X[N] = 0
          const cplx<T> w = cconj(dtw[k]);
          const T a1 = ra[k], a2 = k ? ra[N - k] : T(0);
          const T b1 = r1 < rows ? rb[k] : T(0), b2 = (r1 < rows && k) ? rb[N - k] : T(0);
          xa = cmul(w, cplx<T>{a1, -a2});
          xb = cmul(w, cplx<T>{b1, -b2});
        }
        z[q] = {xa.x - xb.y, xa.y + xb.x};   // XA + i XB
      }
    }
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int t = t0 + q * blockDim.x;
      if (t < nl * N) {
        const int l = t / N, k = t - l * N;
        A[l * N + k] = z[q];
      }
    }
  }
  __syncthreads();
  cplx<T>* z = fft_any<T, PL>(A, B, N, N, nl, rad, tw, true);
  const T inv_n = T(1) / T(N);
  for (int t = threadIdx.x; t < nl * N; t += blockDim.x) {
    const int l = t / N, i = t - l * N;
    const int r0 = 2 * (line0 + l), r1 = r0 + 1;
    int src = i;
    if (mode == 1) src = (i & 1) ? N - 1 - (i >> 1) : (i >> 1);
    const cplx<T> v = z[l * N + src];
    data[(size_t)r0 * N + i] = v.x * inv_n;
    if (r1 < rows) data[(size_t)r1 * N + i] = v.y * inv_n;
  }
}

// ---------------------------------------------------------------------------
// z transforms (3-D, periodic z): complex lines of slot pairs (2m, 2m+1) along z.
template <typename T, int PL>
__global__ void __launch_bounds__(256) zfwd_kernel(T* __restrict__ data, int nx, int ny, int Nrt, int ppb, Radices rad,
                            const cplx<T>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  const int N = PL >= 2 ? PL : Nrt;
  cplx<T>* A = reinterpret_cast<cplx<T>*>(smem_raw);
  const int P = N + 1;   // padded line pitch: lines start in different banks
  cplx<T>* B = A + (size_t)ppb * P;
  const int j = blockIdx.y;
  const int pair0 = blockIdx.x * ppb;
  const int np = min(ppb, nx / 2 - pair0);
  const size_t plane = (size_t)nx * ny;
  T* base = data + (size_t)nx * j + 2 * pair0;
  if constexpr (PL >= 2) {
    // ppb == kMaxLines: thread = (slot sl of the block's 32, z row k0 + 8 q)
    const int sl = threadIdx.x & 31, k0 = threadIdx.x >> 5;
    const bool act = sl < 2 * np;
    constexpr int NQ = PL / 8;
    T v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = act ? base[plane * (k0 + 8 * q) + sl] : T(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) reinterpret_cast<T*>(&A[(sl >> 1) * P + k0 + 8 * q])[sl & 1] = v[q];
  } else {
    constexpr int KB = 8;
    for (int t0 = threadIdx.x; t0 < 2 * np * N; t0 += KB * blockDim.x) {
      T v[KB];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int t = t0 + q * blockDim.x;
        v[q] = T(0);
        if (t < 2 * np * N) {
          const int k = t / (2 * np), sl = t - k * (2 * np);
          v[q] = base[plane * k + sl];
        }
      }
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int t = t0 + q * blockDim.x;
        if (t < 2 * np * N) {
          const int k = t / (2 * np), sl = t - k * (2 * np);
          reinterpret_cast<T*>(&A[(sl >> 1) * P + k])[sl & 1] = v[q];
        }
      }
    }
  }
  __syncthreads();
  cplx<T>* Z = fft_any<T, PL>(A, B, N, P, np, rad, tw, false);
  const int tstride = PL >= 2 ? 32 : 2 * np;   // PL >= 2: the thread's slot is fixed
  for (int t = threadIdx.x; t < tstride * N; t += blockDim.x) {
    const int p = t / tstride, sl = t - p * tstride;
    if (sl >= 2 * np) continue;
    const int line = sl >> 1;
    const int m = pair0 + line;
    T out;
    if (m > 0) {
      const cplx<T> z = Z[line * P + p];
      out = (sl & 1) ? z.y : z.x;
    } else {
      // pair 0 holds two real sequences: split into two real-packed z spectra
      const int l = p == 0 ? 0 : (p == 1 ? N / 2 : p >> 1);
      const bool im = p >= 2 && (p & 1);
      const cplx<T> z = Z[line * P + l], zr = Z[line * P + (l == 0 ? 0 : N - l)];
      if ((sl & 1) == 0) out = im ? T(0.5) * (z.y - zr.y) : T(0.5) * (z.x + zr.x);
      else out = im ? T(0.5) * (zr.x - z.x) : T(0.5) * (z.y + zr.y);
    }
    base[plane * p + sl] = out;
  }
}

template <typename T, int PL>
__global__ void __launch_bounds__(256) zinv_kernel(T* __restrict__ data, int nx, int ny, int Nrt, int ppb, Radices rad,
                            const cplx<T>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  const int N = PL >= 2 ? PL : Nrt;
  cplx<T>* A = reinterpret_cast<cplx<T>*>(smem_raw);
  const int P = N + 1;   // padded line pitch: lines start in different banks
  cplx<T>* B = A + (size_t)ppb * P;
  const int j = blockIdx.y;
  const int pair0 = blockIdx.x * ppb;
  const int np = min(ppb, nx / 2 - pair0);
  const size_t plane = (size_t)nx * ny;
  T* base = data + (size_t)nx * j + 2 * pair0;
  // pair 0 (first block only) arrives as two real-packed spectra and is rebuilt
  // below; every other line is loaded straight into A
  cplx<T>* dst = pair0 == 0 ? B : A;
  if constexpr (PL >= 2) {
    const int sl = threadIdx.x & 31, k0 = threadIdx.x >> 5;
    const bool act = sl < 2 * np;
    constexpr int NQ = PL / 8;
    T v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = act ? base[plane * (k0 + 8 * q) + sl] : T(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) reinterpret_cast<T*>(&dst[(sl >> 1) * P + k0 + 8 * q])[sl & 1] = v[q];
  } else {
    constexpr int KB = 8;
    for (int t0 = threadIdx.x; t0 < 2 * np * N; t0 += KB * blockDim.x) {
      T v[KB];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int t = t0 + q * blockDim.x;
        v[q] = T(0);
        if (t < 2 * np * N) {
          const int k = t / (2 * np), sl = t - k * (2 * np);
          v[q] = base[plane * k + sl];
        }
      }
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int t = t0 + q * blockDim.x;
        if (t < 2 * np * N) {
          const int k = t / (2 * np), sl = t - k * (2 * np);
          reinterpret_cast<T*>(&dst[(sl >> 1) * P + k])[sl & 1] = v[q];
        }
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < np * N; t += blockDim.x) {
    const int line = t / N, l = t - line * N;
    const int m = pair0 + line;
    if (m > 0) {
      if (pair0 == 0) A[line * P + l] = B[line * P + l];
    } else {
      // rebuild Z = Y0 + i Y1 from the two real-packed spectra held in .x (slot 0) and .y (slot 1)
      cplx<T> y0, y1;
      const cplx<T>* Q = B + line * P;
      if (l == 0) { y0 = {Q[0].x, T(0)}; y1 = {Q[0].y, T(0)}; }
      else if (2 * l == N) { y0 = {Q[1].x, T(0)}; y1 = {Q[1].y, T(0)}; }
      else if (2 * l < N) { y0 = {Q[2 * l].x, Q[2 * l + 1].x}; y1 = {Q[2 * l].y, Q[2 * l + 1].y}; }
      else { const int q = N - l; y0 = {Q[2 * q].x, -Q[2 * q + 1].x}; y1 = {Q[2 * q].y, -Q[2 * q + 1].y}; }
      A[line * P + l] = {y0.x - y1.y, y0.y + y1.x};
    }
  }
  __syncthreads();
  cplx<T>* z = fft_any<T, PL>(A, B, N, P, np, rad, tw, true);
  const T inv_n = T(1) / T(N);
  if constexpr (PL >= 2) {
    const int sl = threadIdx.x & 31, k0 = threadIdx.x >> 5;
    if (sl < 2 * np) {
#pragma unroll 4
      for (int q = 0; q < PL / 8; ++q) {
        const int k = k0 + 8 * q;
        const cplx<T> v = z[(sl >> 1) * P + k];
        base[plane * k + sl] = ((sl & 1) ? v.y : v.x) * inv_n;
      }
    }
  } else {
    for (int t = threadIdx.x; t < 2 * np * N; t += blockDim.x) {
      const int k = t / (2 * np), sl = t - k * (2 * np);
      const cplx<T> v = z[(sl >> 1) * P + k];
      base[plane * k + sl] = ((sl & 1) ? v.y : v.x) * inv_n;
    }
  }
}

// ---------------------------------------------------------------------------
// y solve: one thread per (slot s, z position t) column; FP64 Thomas with
// factors e_j = 1 / beta_j and c'_j tabulated per eigenvalue index.
struct YArgs {
  int nx, ny, nz, dim, xmode, nmx, nlz, cyclic;
  const double* a;       // a_j
  const double* E;       // [ny][nlam]
  const double* CP;
  const double* ZV;      // right spikes v_j  [ny][nlam]
  const double* WV;      // left spikes w_j   [ny][nlam]
  const double* MI;      // inverse interface matrices [NRED * NRED][nlam]
  const double* hy;      // cell widths (zero-mode mean)
  double hysum;          // sum of the cell widths
  int pitch;             // 8-column blocks: E, CP, ZV, WV are [nlam][pitch] (eigenvalue-major)
  unsigned* status;      // device status word (bit 0: a staged copy wait gave up)
};

__device__ __forceinline__ int lam_index(const YArgs& A, int s, int t) {
  int mx;
  if (A.xmode == 1) mx = s;
  else mx = s == 0 ? 0 : (s == 1 ? A.nx / 2 : (s >> 1));
  if (A.dim == 2) return mx;
  int l = (s >= 2 || A.xmode == 1) ? t : (t == 0 ? 0 : (t == 1 ? A.nz / 2 : (t >> 1)));
  const int lz = min(l, A.nz - l);
  return lz * A.nmx + mx;   // tables are [j][lz][mx]: consecutive slots read consecutive entries
}

// Partitioned (SPIKE) solve: every column is split into NSEG segments of
// about ny / NSEG rows solved concurrently by NSEG threads (NSEG = 4, or 8 for
// ny >= 192 and for grids with too few columns to occupy every SM twice).  Each segment's
// local factors (e_j = 1 / beta_j, c'_j) and its two spikes (the response to
// its coupling with the neighbouring segments, v_j and w_j) are tabulated per
// eigenvalue on the host, so one step of the solve is
//   1. y = A_p^-1 d on each segment (FP64 Thomas, local factors)
//   2. the 2 NSEG interface values X_p = x[first of p], Y_p = x[last of p] from
//        X_p + v_f X_{p+1} + w_f Y_{p-1} = y_f,   Y_p + v_l X_{p+1} + w_l Y_{p-1} = y_l
//      (periodic y couples the last and first segments).  That 2 NSEG system
//      depends on the eigenvalue only: its inverse is tabulated on the host and
//      the NSEG threads of a column each form two of its rows' products in FP64
//   3. x_j = y_j - v_j X_{p+1} - w_j Y_{p-1} on every row.
// The singular zero mode pins x_0 = 0 (e_0 = 0 in its table) and is shifted to
// zero hy-weighted mean afterwards.
constexpr int YCOLS = 32;   // columns per block (8, with staged tables, on grids with few columns)

// YC = 8 (grids with few columns) also stages the block's table columns and the
// couplings a_j in shared memory, so that the sequential sweeps wait on shared
// rather than global loads.
template <typename T, int NSEG, int YC>
__global__ void __launch_bounds__(YC * NSEG) ysolve_kernel(T* __restrict__ data, const YArgs A) {
  constexpr int NRED = 2 * NSEG;
  constexpr bool STG = YC == 8;
  extern __shared__ __align__(16) double sm[];
  const int ny = A.ny;
  double* D = sm;                                  // [ny][YC] data tile, then y, then x
  double* Z = D + (size_t)ny * YC;              // [YC][NRED] interface values
  double* R = Z + YC * NRED;                    // [YC][NSEG] mean partial sums
  double* ST = R + YC * NSEG;                   // STG: [4 tables][YC][ny + 1], then a_j [ny]
  const int tx = threadIdx.x, p = threadIdx.y;
  const int tid = tx + YC * p;
  const int s0 = blockIdx.x * YC;
  const int t = blockIdx.y;
  const int s = s0 + tx;
  const int ncol = min(YC, A.nx - s0);
  const int nlam = A.nmx * A.nlz;
  T* tile = data + s0 + (size_t)A.nx * A.ny * t;
  const size_t rs = (size_t)A.nx;
  // tile in (unrolled for the short columns of the 8- and 16-segment forms; the 4-segment
  // form of large 3-D grids runs faster with the plain loop)
  if constexpr (NSEG >= 8) {
#pragma unroll 8
    for (int e = tid; e < ny * YC; e += YC * NSEG) {
      const int j = e / YC, c = e - j * YC;
      D[e] = c < ncol ? (double)tile[rs * j + c] : 0.0;
    }
  } else {
    for (int e = tid; e < ny * YC; e += YC * NSEG) {
      const int j = e / YC, c = e - j * YC;
      D[e] = c < ncol ? (double)tile[rs * j + c] : 0.0;
    }
  }
  // STG: the block's 8 table columns and a_j land in shared memory by bulk copies while the tile loads
  const int sp = A.pitch + 2;   // padded slot pitch (16-byte multiple, odd in 16-byte units)
  __shared__ uint64_t tbar;
  bool tok = true;
  if constexpr (STG) {
    if (tid == 0) {
      mbar_init(&tbar, 1);
      mbar_init_fence();
      const uint32_t col = (uint32_t)A.pitch * sizeof(double);
      mbar_expect_tx(&tbar, (4 * YC + 1) * col);
      const double* tabs[4] = {A.E, A.CP, A.ZV, A.WV};
      for (int c = 0; c < YC; ++c) {
        const int lc = s0 + c < A.nx ? lam_index(A, s0 + c, t) : 0;
        for (int q = 0; q < 4; ++q) bulk_g2s(ST + (q * YC + c) * sp, tabs[q] + (size_t)lc * A.pitch, col, &tbar);
      }
      bulk_g2s(ST + 4 * YC * sp, A.a, col, &tbar);
    }
  }
  __syncthreads();
  if constexpr (STG) tok = mbar_wait(&tbar, 0);
  const bool act = s < A.nx;
  const int li = act ? lam_index(A, s, t) : 0;
  const int r0 = (p * ny) / NSEG, r1 = ((p + 1) * ny) / NSEG;
  const double* E = A.E + li;
  const double* CP = A.CP + li;
  const double* V = A.ZV + li;    // right spikes
  const double* W = A.WV + li;    // left spikes
  // table entries of this thread's column (shared-memory copies when staged)
  auto fE = [&](int j) -> double {
    if constexpr (STG) return ST[(0 * YC + tx) * sp + j];
    else return __ldg(E + (size_t)j * nlam);
  };
  auto fCP = [&](int j) -> double {
    if constexpr (STG) return ST[(1 * YC + tx) * sp + j];
    else return __ldg(CP + (size_t)j * nlam);
  };
  auto fV = [&](int j) -> double {
    if constexpr (STG) return ST[(2 * YC + tx) * sp + j];
    else return __ldg(V + (size_t)j * nlam);
  };
  auto fW = [&](int j) -> double {
    if constexpr (STG) return ST[(3 * YC + tx) * sp + j];
    else return __ldg(W + (size_t)j * nlam);
  };
  auto fa = [&](int j) -> double {
    if constexpr (STG) return ST[4 * YC * sp + j];
    else return __ldg(A.a + j);
  };
  double* col = D + tx;
  constexpr int U = 8;            // table rows fetched ahead of their use
  if (act && r1 > r0) {
    // 1. segment Thomas
    double prev = 0.0;
    int j = r0;
    for (; j + U <= r1; j += U) {
      double e[U], a[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        e[q] = fE(j + q);
        a[q] = fa(j + q);
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const double d = col[(j + q) * YC];
        prev = (j + q == r0) ? d * e[q] : (d - a[q] * prev) * e[q];
        col[(j + q) * YC] = prev;
      }
    }
    for (; j < r1; ++j) {
      const double d = col[j * YC];
      prev = (j == r0) ? d * fE(j) : (d - fa(j) * prev) * fE(j);
      col[j * YC] = prev;
    }
    double x = prev;
    j = r1 - 2;
    for (; j - U + 1 >= r0; j -= U) {
      double c[U];
#pragma unroll
      for (int q = 0; q < U; ++q) c[q] = fCP(j - q);
#pragma unroll
      for (int q = 0; q < U; ++q) {
        x = col[(j - q) * YC] - c[q] * x;
        col[(j - q) * YC] = x;
      }
    }
    for (; j >= r0; --j) {
      x = col[j * YC] - fCP(j) * x;
      col[j * YC] = x;
    }
  }
  __syncthreads();
  // 2. interface values: z = Minv b, b = (y[first], y[last]) of every segment
  if (act) {
    double b[NRED];
#pragma unroll
    for (int g = 0; g < NSEG; ++g) {
      const int a0 = (g * ny) / NSEG, a1 = ((g + 1) * ny) / NSEG;
      b[2 * g] = a1 > a0 ? col[a0 * YC] : 0.0;
      b[2 * g + 1] = a1 > a0 ? col[(a1 - 1) * YC] : 0.0;
    }
    double* z = Z + tx * NRED;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = 2 * p + h;
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < NRED; ++q) v += __ldg(A.MI + (size_t)(r * NRED + q) * nlam + li) * b[q];
      z[r] = v;
    }
  }
  __syncthreads();
  // 3. spike correction
  double part = 0.0;
  if (act && r1 > r0) {
    const bool cyc = A.cyclic != 0;
    const double* z = Z + tx * NRED;
    const int gn = p + 1 < NSEG ? p + 1 : 0, gp = p > 0 ? p - 1 : NSEG - 1;
    const double Xn = (p + 1 < NSEG || cyc) ? z[2 * gn] : 0.0;
    const double Yp = (p > 0 || cyc) ? z[2 * gp + 1] : 0.0;
    for (int j = r0; j < r1; ++j) {
      const double r = col[j * YC] - fV(j) * Xn - fW(j) * Yp;
      col[j * YC] = r;
      if (li == 0) part += r * __ldg(A.hy + j);
    }
  }
  // singular zero mode: shift to zero hy-weighted mean
  if (li == 0 && act) R[tx * NSEG + p] = part;
  __syncthreads();
  if (li == 0 && act && r1 > r0) {
    double sx = 0.0;
    for (int g = 0; g < NSEG; ++g) sx += R[tx * NSEG + g];
    const double mean = sx / A.hysum;
    for (int j = r0; j < r1; ++j) col[j * YC] -= mean;
  }
  __syncthreads();
  if constexpr (NSEG >= 8) {
#pragma unroll 8
    for (int e = tid; e < ny * YC; e += YC * NSEG) {
      const int j = e / YC, c = e - j * YC;
      if (c < ncol) tile[rs * j + c] = (T)D[e];
    }
  } else {
    for (int e = tid; e < ny * YC; e += YC * NSEG) {
      const int j = e / YC, c = e - j * YC;
      if (c < ncol) tile[rs * j + c] = (T)D[e];
    }
  }
  if (!tok) atomicOr(A.status, 1u);   // the staged tables never arrived: this block's columns are invalid
}

// ---------------------------------------------------------------------------
// y solve for grids with many columns: twisted (two-sided) factorisation, two
// threads per column and no partition corrections.
//
// The chain of rows 0..L-1 (L = ny; with periodic y, L = ny - 1 and row ny - 1
// is bordered off, below) is eliminated from both ends at once: the upper
// thread runs forward elimination over rows 0..k, the lower thread backward
// elimination over rows L-1..k+1,
//   g_j = d_j + M_j g_{j-1}   (upper),      h_j = d_j + M_j h_{j+1}   (lower),
// which leaves the 2x2 system of rows k, k+1, solved with its tabulated
// inverse P after one shuffle between the two threads; each thread then
// substitutes outward,
//   x_j = E_j g_j + C_j x_{j+1}   (upper),  x_j = E_j h_j + C_j x_{j-1}   (lower).
// That is one FP64 multiply-add per row forward and a multiply plus a
// multiply-add backward: the FP64 work of a plain Thomas solve, spread over
// twice the threads.  M, E, C are tabulated per eigenvalue (M and C negated).
// With FP32 fields the backward pass carries y_j = x_j / sigma_j instead
// (sigma_j = E_j; 1 at each thread's last row, 0 at the zero mode's pinned row):
//   y_j = g_j + C'_j y_{j+1},   C'_j = C_j sigma_{j+1} / sigma_j,
// one multiply-add per row; sigma is applied in FP32 as the result is narrowed
// (x = sigma y: two FP32 roundings of the FP64 solution instead of one).
//
// Periodic y (cyclic): with xi = x_{ny-1}, rows 0..ny-2 read A'' x' = d' - xi u,
// u the coupling column of x_{ny-1}; so x' = y - xi z with A'' y = d' (the solve
// above) and z = A''^-1 u (tabulated), and row ny-1 gives
//   xi = (d_{ny-1} - S0 y_0 - S1 y_{ny-2}) S2,   S2 = 1 / (b_{ny-1} - S0 z_0 - S1 z_{ny-2}),
// S0, S1 its couplings to x_0 and x_{ny-2}: one more multiply-add per row where
// z matters (FP32 fields: z / sigma, and S0, S1 times sigma).  z decays geometrically away from the chain's ends (faster for the
// larger x/z eigenvalues); a warp corrects the leading positions of its threads
// up to the last one where some column's |z| exceeds 2^-56 of its largest
// (tabulated per eigenvalue, K), beyond which the correction is below FP64
// rounding of the solution's scale.
//
// Positions: both threads of a column own R = ceil(L / 2) consecutive
// positions and sweep them in the same direction.  The upper thread's are rows
// 0..R-1; the lower thread's start at position R with, when L is odd, one
// inert slot (multiplier 0, E = 1, C = 0, z = 0) that holds the bordered row
// ny - 1 on periodic y, followed by rows L-1 down to R.  Shared memory and the
// tables are then read at fixed strides from one base, with no per-row bounds.
// The tables are position-major ([2 U zero rows, 2 R positions, 2 U zero
// rows][eigenvalues]): the 16 threads of a half-warp read 8 consecutive
// eigenvalues of one position, one coalesced 64-byte segment (one column per
// eigenvalue instead scatters each such read over 16 lines and halves the
// sweep rate).
//
// B300's FP64 pipe (one warp instruction per ~73 cycles per SM sub-partition,
// conversions included) bounds the sweeps, which need 2 FP64 operations per
// cell with FP32 fields (3 with FP64 fields; one more with periodic y where z
// matters).  The block therefore splits its warps: four "sweep" warps run the
// chains and issue little besides FP64, while four helper warps widen the FP32
// spectrum to FP64 with integer field arithmetic (fpconv.cuh) as its row groups
// arrive by tensor-map copies, releasing each group to the sweeps on an
// mbarrier, then stage sigma in the freed FP32 tile, and narrow the solution
// chunk by chunk as the sweeps finish it: the chunks nearest the middle first,
// during the outward pass where no z reaches them.
//
// The singular zero mode pins x_0 = 0 through its tables (E_0 = C_0 = 0,
// M_1 = 0, no coupling to row 0) and is shifted to zero hy-weighted mean (with
// FP32 fields the shift, a constant invisible to the pressure gradient, is
// applied after narrowing).
//
// 3-D blocks are ordered so that the z positions t and nz - t, which share every
// eigenvalue, run next to each other.
struct YTwArgs {
  int nx, ny, nz, dim, xmode, nmx, nlz;
  int L, R;              // chain rows 0..L-1; positions per thread R = ceil(L / 2)
  int nlp;               // table row pitch (eigenvalues, even, >= nlam + 2)
  int bulk;              // rows move by bulk copies (16-byte aligned rows and widths)
  int tiled;             // FP32: the tile arrives as 32-row boxes of the tensor map (row order)
  const double* M;       // [2 U + 2 R + 2 U][nlp] forward multipliers (negated), position-major
  const double* E;       // inverse pivots, same layout (FP64 fields)
  const double* C;       // outward multipliers (negated; FP32 fields: of the scaled pass)
  const float* sig;      // FP32 fields: sigma per position (x = sigma y), same layout
  const double* sig0;    // FP32 fields: sigma of the zero mode's column [2 R]
  const double* Z;       // cyclic: z = A''^-1 u
  const double* P;       // [nlam][4] inverse of the middle 2x2 system
  const double* S;       // [nlam][4] cyclic: S0, S1, S2
  const int* K;          // [nlam] cyclic: positions per thread (from its first) where z matters
  const double* hy;      // cell widths (zero-mode mean)
  double hysum_inv;      // 1 / their sum
  int hy_uniform;        // uniform y cells (the mean is then unweighted)
  int gauge;             // shift the zero mode's column to zero hy-weighted mean
  unsigned* status;      // device status word (bit 0: a bulk copy or group wait gave up)
  int xblk0;             // first block of columns along x (blockIdx.x + xblk0)
};

constexpr int kTwU = kTwChunk;   // rows per chunk of the twisted solve (tables fetched a chunk ahead)

__device__ __forceinline__ int lam_of(int nx, int nz, int dim, int xmode, int nmx, int s, int t) {
  int mx;
  if (xmode == 1) mx = s;
  else mx = s == 0 ? 0 : (s == 1 ? nx / 2 : (s >> 1));
  if (dim == 2) return mx;
  const int l = (s >= 2 || xmode == 1) ? t : (t == 0 ? 0 : (t == 1 ? nz / 2 : (t >> 1)));
  return min(l, nz - l) * nmx + mx;
}

template <typename T>
__device__ __forceinline__ double widen(T v) {
  if constexpr (sizeof(T) == 4) return fsconv_widen(v);
  else return v;
}
template <typename T>
__device__ __forceinline__ T narrow(double v) {
  if constexpr (sizeof(T) == 4) return fsconv_narrow(v);
  else return v;
}

template <typename T>
size_t ytwist_smem(int ny, int w) {
  const size_t np = (size_t)ny + 1;   // 2 R positions <= ny + 1
  return np * w * (sizeof(double) + (sizeof(T) == 4 ? sizeof(T) : 0)) + 128;   // + alignment slack
}

constexpr int kTwBoxRows = 16;   // rows per tensor-map box of the twisted solve's tile (one chunk)

template <typename T, bool CYC, int W>
__global__ void __launch_bounds__(4 * W, W == 32 ? 4 : 2) ytwist_kernel(T* __restrict__ data, const YTwArgs A,
                                                          const __grid_constant__ CUtensorMap tmap) {
  constexpr bool F32 = sizeof(T) == 4;
  constexpr int U = kTwU;
  constexpr int NG = 4;                          // tile row groups: offsets [16 g, 16 g + 16), the last open
  constexpr int NS = 2 * W;                      // sweep threads (warps 0 .. W / 16 - 1)
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(128) unsigned char ytw_smem[];
  // 128-byte aligned base (tensor-map box destinations); the launch adds 128 bytes for it
  unsigned char* ytw_raw = ytw_smem + ((128u - (smem_u32(ytw_smem) & 127u)) & 127u);
  const int ny = A.ny, L = A.L, R = A.R;
  const int NP = 2 * R;                          // positions
  const bool odd = (L & 1) != 0;                 // the lower thread's first position is the inert slot
  double* sg = reinterpret_cast<double*>(ytw_raw);   // [NP][W] FP64, position order
  T* st = F32 ? reinterpret_cast<T*>(ytw_raw + (size_t)(ny + 1) * W * sizeof(double)) : reinterpret_cast<T*>(sg);
  constexpr int ND = 20;                         // output chunks of 16 positions (R <= 293 rows per thread)
  constexpr int NB = 20;                         // tensor-map boxes of kTwBoxRows rows (ny <= 320)
  __shared__ uint64_t bulkbar[NB], widebar[NB], donebar[ND];
  __shared__ uint64_t stfree;                    // tiled FP32: the sweeps are done with the stage buffer
  __shared__ uint64_t sigbar;                    // FP32: sigma is staged
  // 32-column blocks: the sweep and helper warps trade places in every other block, so that
  // the sweeps of neighbouring blocks on an SM sit on different sub-partitions (FP64 pipes)
  const int tid = (W == 32 && ((blockIdx.x + blockIdx.y) & 1)) ? (int)(threadIdx.x ^ (2 * W)) : (int)threadIdx.x;
  const int lane = tid & 31;
  const int s0 = (blockIdx.x + A.xblk0) * W;
  const int ncol = min(W, A.nx - s0);
  int t = 0;
  if (A.dim == 3) {
    const int b = blockIdx.y;
    t = (b & 1) ? A.nz - ((b + 1) >> 1) : (b >> 1);
  }
  const size_t rs = (size_t)A.nx;
  T* tile = data + (size_t)A.nx * ny * t + s0;
  // position of row j
  auto pos = [&](int j) { return j < R ? j : (j < L ? R + (odd ? 1 : 0) + (L - 1 - j) : R); };
  // row at position p (-1: the lower thread's inert slot on walls)
  auto rowof = [&](int p) { return p < R ? p : (odd && p == R ? (CYC ? ny - 1 : -1) : L - 1 - (p - R - (odd ? 1 : 0))); };
  // group of position p: its offset from its thread's first position, in chunks of 16
  auto pgroup = [&](int p) { return min(NG - 1, (p < R ? p : p - R) >> 4); };
  const uint32_t rb = (uint32_t)(ncol * sizeof(T));
  const int nchunk = (R + U - 1) / U;
  const int nbox = (ny + kTwBoxRows - 1) / kTwBoxRows, nlev = (nbox + 1) / 2;
  // the block holding the zero mode (column 0), when its gauge is to be set
  const bool zb = A.gauge && s0 == 0 && (A.dim == 2 || t == 0);
  bool ok = true;
  if (tid == 0) {
    for (int g = 0; g < NB; ++g) {
      mbar_init(&bulkbar[g], 1);
      mbar_init(&widebar[g], W / 16);            // one arrival per helper warp
    }
    for (int c = 0; c < ND; ++c) mbar_init(&donebar[c], W / 16);   // one arrival per sweep warp
    mbar_init(&stfree, W / 16);
    mbar_init(&sigbar, W / 16);                  // one arrival per helper warp
    mbar_init_fence();
  }
  __syncthreads();
  if (tid < NS) {
    // ---------------- sweep threads: two per column ----------------
    const int half = lane >> 4;
    const int cb = (tid >> 5) * 16 + (lane & 15);
    const int s = s0 + cb;
    const bool act = cb < ncol;
    const int li = act ? lam_of(A.nx, A.nz, A.dim, A.xmode, A.nmx, s, t) : 0;
    const int P0 = half ? R : 0;
    const size_t nl = (size_t)A.nlp;
    const size_t tb = (size_t)(2 * U + P0) * nl + li;
    const double* __restrict__ Mt = A.M + tb;
    // one buffer per table: a chunk's entries are consumed in order and each slot refilled with
    // the entry a chunk further on
    double mb[U];
#pragma unroll
    for (int q = 0; q < U; ++q) mb[q] = __ldg(Mt + q * nl);   // tables do not depend on the predecessor
    // periodic y: positions per thread (from its first) where z matters, for this column
    const int kwl = CYC && act ? __ldg(A.K + li) : 1;
    double* gp = sg + P0 * W + cb;
    // 1. elimination towards the middle; chunk c waits for its rows
    if (F32 && A.tiled) {
      // chunk 0 is exactly the rows of box 0 (upper thread) or box 1 (lower): widened here, by
      // the thread that eliminates them, as soon as the box lands
      ok &= mbar_wait_idle(&bulkbar[half], 0);
      uint32_t sp = 0;
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int j = rowof(P0 + q);
        uint32_t whi, wlo;
        fsconv_widen_fast(act && j >= 0 ? __float_as_uint((float)st[j * W + cb]) : 0u, &whi, &wlo, &sp);
        gp[q * W] = __hiloint2double((int)whi, (int)wlo);
      }
      if (__any_sync(FULL, sp)) {
#pragma unroll
        for (int q = 0; q < U; ++q) {
          const int j = rowof(P0 + q);
          gp[q * W] = act && j >= 0 ? widen<T>(st[j * W + cb]) : 0.0;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&stfree);      // the stage buffer's rows of chunk 0 are read
    }
    double gv = 0.0;
    for (int i0 = 0; i0 < R; i0 += U) {
      // tiled: level l (two boxes, kTwBoxRows rows from each end) holds chunk l; chunk 0 is ours
      if (!A.tiled) ok &= mbar_wait_idle(&widebar[min(NG - 1, i0 >> 4)], 0);
      else if (i0 > 0) ok &= mbar_wait_idle(&widebar[min(nlev - 1, i0 / kTwBoxRows)], 0);
      if (i0 + U <= R) {
        // the chunk's values first, the chain in registers, the stores after: no store waits on
        // the chain ahead of the next chunk's loads
        double d[U], m[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
          d[q] = gp[(i0 + q) * W];
          m[q] = mb[q];
          mb[q] = __ldg(Mt + (i0 + U + q) * nl);
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
          gv = fma(m[q], gv, d[q]);
          d[q] = gv;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) gp[(i0 + q) * W] = d[q];
      } else {
#pragma unroll
        for (int q = 0; q < U; ++q) {
          if (i0 + q < R) {
            gv = fma(mb[q], gv, gp[(i0 + q) * W]);
            gp[(i0 + q) * W] = gv;
          }
        }
      }
    }
    // 2. the middle rows (each thread's last position)
    const double oth = __shfl_xor_sync(FULL, gv, 16);
    const double gk = half ? oth : gv, hk = half ? gv : oth;
    const double* Pt = A.P + (size_t)li * 4 + 2 * half;
    double xv = fma(__ldg(Pt), gk, __ldg(Pt + 1) * hk);
    gp[(R - 1) * W] = xv;
    // 3. outward substitution, positions descending (FP32 fields: y = x / sigma, one multiply-add
    // per row; FP64 fields: x = E g + C x_next)
    if constexpr (CYC) {
      // the cyclic correction's first table entries into L2 meanwhile (its start waits on them)
#pragma unroll
      for (int q = 0; q < U; ++q) prefetch_l2(A.Z + tb + q * nl);
      prefetch_l2(A.S + (size_t)li * 4);
    }
    // periodic y: the chunks the cyclic correction touches in some column of this warp; the
    // outward pass hands every later chunk to the helpers as soon as it is final
    const int nkw = CYC ? (__reduce_max_sync(FULL, kwl) + U - 1) / U : 0;
    {
      const double* __restrict__ Et = A.E + tb;
      const double* __restrict__ Ct = A.C + tb;
      double eb[F32 ? 1 : U], cbuf[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        if constexpr (!F32) eb[q] = __ldg(Et + (R - 2 - q) * (ptrdiff_t)nl);
        cbuf[q] = __ldg(Ct + (R - 2 - q) * (ptrdiff_t)nl);
      }
      int next = nchunk - 1;                     // highest output chunk not yet released
      for (int i0 = R - 2; i0 >= 0; i0 -= U) {
        if (i0 + 1 >= U) {
          // products E g first (independent), the chain in registers, the stores after
          double v[U], c2[U];
#pragma unroll
          for (int q = 0; q < U; ++q) {
            if constexpr (F32) {
              v[q] = gp[(i0 - q) * W];
            } else {
              v[q] = eb[q] * gp[(i0 - q) * W];
              eb[q] = __ldg(Et + (i0 - U - q) * (ptrdiff_t)nl);
            }
            c2[q] = cbuf[q];
            cbuf[q] = __ldg(Ct + (i0 - U - q) * (ptrdiff_t)nl);
          }
#pragma unroll
          for (int q = 0; q < U; ++q) {
            xv = fma(c2[q], xv, v[q]);
            v[q] = xv;
          }
#pragma unroll
          for (int q = 0; q < U; ++q) gp[(i0 - q) * W] = v[q];
        } else {
#pragma unroll
          for (int q = 0; q < U; ++q) {
            if (q <= i0) {
              double eg;
              if constexpr (F32) eg = gp[(i0 - q) * W];
              else eg = eb[q] * gp[(i0 - q) * W];
              xv = fma(cbuf[q], xv, eg);
              gp[(i0 - q) * W] = xv;
            }
          }
        }
        {
          // positions max(i0 - U + 1, 0) .. R - 1 are final (periodic y: where no z reaches them):
          // hand their chunks to the helpers
          const int lowest = max(i0 - U + 1, 0);
          __syncwarp();
          while (next >= nkw && U * next >= lowest) {
            if (lane == 0) mbar_arrive(&donebar[next]);
            --next;
          }
        }
      }
      if constexpr (!CYC) {
        __syncwarp();
        for (; next >= 0; --next)
          if (lane == 0) mbar_arrive(&donebar[next]);
      }
    }
    pdl_trigger();
    if constexpr (CYC) {
      // 4. the bordered row ny - 1 (the lower thread's inert slot, still d_{ny-1}), then x = y - xi z
      const double yl_own = gp[W];                       // lower: row L - 1 at its second position
      const double o2 = __shfl_xor_sync(FULL, half ? yl_own : xv, 16);
      const double y0 = half ? o2 : xv, yl = half ? yl_own : o2;
      const double dl = __shfl_xor_sync(FULL, gp[0], 16);  // the lower's inert slot, seen by the upper
      const double dlast = half ? gp[0] : dl;
      const double* St = A.S + (size_t)li * 4;
      const double xi = fma(-__ldg(St + 1), yl, fma(-__ldg(St), y0, dlast)) * __ldg(St + 2);
      const double* __restrict__ Zt = A.Z + tb;
      // the chunks some z of this warp's columns reaches (the later ones went to the helpers in the
      // outward pass), corrected from the middle outward: the helpers narrow in the same order
      double zv[U];
#pragma unroll
      for (int q = 0; q < U; ++q) zv[q] = __ldg(Zt + ((nkw - 1) * U + q) * nl);
      for (int c = nkw - 1; c >= 0; --c) {
        const int i0 = c * U;
        double v[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
          v[q] = fma(-xi, zv[q], gp[min(i0 + q, R - 1) * W]);
          zv[q] = __ldg(Zt + (i0 - U + q) * nl);   // the table's zero rows ahead of position 0
        }
        if (half && i0 == 0) v[0] = xi;            // the inert slot becomes x_{ny-1}
#pragma unroll
        for (int q = 0; q < U; ++q)
          if (i0 + q < R) gp[(i0 + q) * W] = v[q];
        __syncwarp();
        if (lane == 0) mbar_arrive(&donebar[c]);   // the helpers narrow this chunk meanwhile
      }
    }
    // 5. the chunk nearest the chain's ends, the last to be final: narrowed by the sweep threads
    // themselves (each its own rows) while the helpers narrow the chunk before it
    {
      const int n0 = min(U, R);
      const bool zc = zb && cb == 0;             // the zero mode's column: kept for its gauge
      float* const ssg = reinterpret_cast<float*>(st) + P0 * W + cb;
      float sv[U];
      if constexpr (F32) {
        ok &= mbar_wait_idle(&sigbar, 0);
#pragma unroll
        for (int q = 0; q < U; ++q) sv[q] = q < n0 ? ssg[q * W] : 0.0f;
      }
      uint32_t sp = 0;
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int j = rowof(P0 + q);
        if (q < n0 && act) {
          const double v = gp[q * W];
          if constexpr (F32) {
            const uint32_t o = fsconv_narrow_fast((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v), &sp);
            const float x = __uint_as_float(o) * sv[q];
            if (zc) ssg[q * W] = x;
            else if (j >= 0) tile[rs * j + cb] = x;
          } else if (!zc && j >= 0) {
            tile[rs * j + cb] = v;
          }
        }
      }
      if constexpr (F32) {
        if (__any_sync(FULL, sp)) {
#pragma unroll
          for (int q = 0; q < U; ++q) {
            const int j = rowof(P0 + q);
            if (q < n0 && act) {
              const float x = fsconv_narrow(gp[q * W]) * sv[q];
              if (zc) ssg[q * W] = x;
              else if (j >= 0) tile[rs * j + cb] = x;
            }
          }
        }
      }
    }
  } else {
    // ---------------- helper threads: tile in, widened, group by group ----------------
    const int h = tid - NS;                      // 0 .. 2 W - 1
    const int hc = h % W, hw = h / W;            // this helper's column and row parity
    if (h >= 32 && !A.tiled) {
      // row copies: the block's table segments into L2 while the tile is in flight (the sweeps'
      // chunk-ahead register fetches then wait on L2, not on DRAM): per position, the eigenvalues
      // of the block's slots at its z wavenumber, one bulk prefetch per table.  (With the tile as
      // tensor-map boxes these requests, sharing the SM's copy engine, delay the boxes more than
      // they save: 0.269 against 0.259 ms per 128^3 step.)
      const int lzb = A.dim == 3 ? min(t, A.nz - t) : 0;
      const int mx0 = A.xmode == 1 ? s0 : s0 / 2;
      const int span = A.xmode == 1 ? W : W / 2 + 1;
      const size_t nl = (size_t)A.nlp;
      const size_t first = ((size_t)lzb * A.nmx + mx0) & ~(size_t)1;
      const uint32_t bytes = (uint32_t)((span + 2) & ~1) * sizeof(double);
      for (int p = h - 32; p < 2 * R; p += NS - 32) {
        const size_t o = (size_t)(2 * U + p) * nl + first;
        bulk_prefetch_l2(A.M + o, bytes);
        if constexpr (!F32) bulk_prefetch_l2(A.E + o, bytes);
        bulk_prefetch_l2(A.C + o, bytes);
        if constexpr (CYC) bulk_prefetch_l2(A.Z + o, bytes);
      }
    }
    pdl_wait();
    if (A.tiled) {
      // boxes of kTwBoxRows rows in row order, from both ends of the column inward (the rows each
      // thread's elimination needs first): box b is the top (b even) or bottom (b odd) box of
      // level b / 2; the stage buffer holds the tile in row order
      auto box_row = [&](int b) {
        const int l = b >> 1;
        return (b & 1) ? max(0, ny - kTwBoxRows * (l + 1)) : kTwBoxRows * l;
      };
      if (h == 0) {
        for (int b = 0; b < nbox; ++b) {
          mbar_expect_tx(&bulkbar[b], (uint32_t)(kTwBoxRows * W * sizeof(T)));
          const int r0 = box_row(b);
          tensor_g2s_3d(st + (size_t)r0 * W, &tmap, s0, r0, t, &bulkbar[b]);
        }
      }
      for (int l = 1; l < nlev; ++l) {   // level 0: the sweep threads' own first chunk
        for (int b = 2 * l; b < min(2 * l + 2, nbox); ++b) {
          ok &= mbar_wait_idle(&bulkbar[b], 0);
          // the rows this box is the first to bring (boxes overlap on ragged columns, and a row
          // the sweeps may already be eliminating in place must not be widened again): with B rows
          // per box the top box of level l owns [B l, min(B l + B, ny - B l)), the bottom box
          // [max(B (l + 1), ny - B (l + 1)), ny - B l)
          const int a0 = (b & 1) ? max(kTwBoxRows * (l + 1), ny - kTwBoxRows * (l + 1)) : kTwBoxRows * l;
          const int a1 = (b & 1) ? ny - kTwBoxRows * l : min(kTwBoxRows * (l + 1), ny - kTwBoxRows * l);
          // this thread: column h % W, rows a0 + h / W + 2 k, by the fast path; a warp that met
          // another value redoes its rows with the general routine
          // (all of a box's loads first: the stage buffer and the FP64 rows share one array, so
          // the compiler would otherwise keep every load behind the previous row's store)
          uint32_t sp = 0, raw[kTwBoxRows / 2];
#pragma unroll
          for (int k = 0; k < kTwBoxRows / 2; ++k) {
            const int j = a0 + hw + 2 * k;
            raw[k] = j < a1 ? __float_as_uint(st[j * W + hc]) : 0u;
          }
#pragma unroll
          for (int k = 0; k < kTwBoxRows / 2; ++k) {
            const int j = a0 + hw + 2 * k;
            if (j < a1) {
              uint32_t whi, wlo;
              fsconv_widen_fast(raw[k], &whi, &wlo, &sp);
              sg[pos(j) * W + hc] = __hiloint2double((int)whi, (int)wlo);
            }
          }
          if (__any_sync(FULL, sp))
            for (int j = a0 + hw; j < a1; j += 2) sg[pos(j) * W + hc] = fsconv_widen(st[j * W + hc]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&widebar[l]);
      }
    } else if (A.bulk) {
      if (h < 32) {
        if (lane < NG) {
          // positions of group g in each half: offsets [16 g, 16 g + 16) (the last group open), minus
          // the lower's inert slot when it holds no row
          const int lo = 16 * lane, hi = lane == NG - 1 ? R : min(R, 16 * lane + 16);
          int rows = 2 * max(0, hi - lo);
          if (odd && !CYC && lane == 0) --rows;
          mbar_expect_tx(&bulkbar[lane], rb * (uint32_t)rows);
        }
        __syncwarp();
        for (int g = 0; g < NG; ++g)
          for (int j = lane; j < ny; j += 32)
            if (pgroup(pos(j)) == g) bulk_g2s(st + (size_t)pos(j) * W, tile + rs * j, rb, &bulkbar[g]);
      }
      for (int g = 0; g < NG; ++g) {
        ok &= mbar_wait(&bulkbar[g], 0);
        // the group's positions: [16 g, ...) in each half
        const int lo = 16 * g, hi = g == NG - 1 ? R : min(R, 16 * g + 16);
        const int n = max(0, hi - lo);
        // this thread: column h % W, rows h / W + 2 k of the group's 2 n (upper n, then lower n)
        for (int r = hw; r < 2 * n; r += 2) {
          const int p = r < n ? lo + r : R + lo + (r - n);
          const bool hole = odd && !CYC && p == R;
          if constexpr (F32) {
            const uint32_t u = (hc < ncol && !hole) ? __float_as_uint(st[p * W + hc]) : 0u;
            uint32_t whi, wlo, sp = 0;
            fsconv_widen_fast(u, &whi, &wlo, &sp);
            sg[p * W + hc] = sp ? fsconv_widen(__uint_as_float(u)) : __hiloint2double((int)whi, (int)wlo);
          } else if (hc >= ncol || hole) {
            sg[p * W + hc] = 0.0;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&widebar[g]);
      }
    } else {
      // plain loads, widened straight into their positions
      for (int e = h; e < NP * W; e += NS) {
        const int p = e / W, c = e - p * W;
        const int j = rowof(p);
        sg[e] = (c < ncol && j >= 0) ? widen<T>(tile[rs * j + c]) : 0.0;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(NS) : "memory");   // every helper's rows are in
      if (lane == 0)
        for (int g = 0; g < NG; ++g) mbar_arrive(&widebar[g]);
    }
    // the solution out, chunk by chunk as the sweeps finish it: narrowed, row-coalesced (the zero
    // mode's column waits for its mean, below)
    const bool zcol = zb && hc == 0, mine = hc < ncol && !zcol;
    // FP32 fields: sigma (x = sigma y) of every position of the block's columns, into the stage
    // buffer once no thread reads the tile there any more ([2 R][W]; 2 R <= ny + 1 rows), by
    // asynchronous copies issued long before the first chunk is narrowed
    float* const ssg = reinterpret_cast<float*>(st);
    if constexpr (F32) {
      if (A.tiled) ok &= mbar_wait_idle(&stfree, 0);
      asm volatile("bar.sync 1, %0;" ::"r"(NS) : "memory");   // every helper is done with the tile
      const int lih = hc < ncol ? lam_of(A.nx, A.nz, A.dim, A.xmode, A.nmx, s0 + hc, t) : 0;
      const float* __restrict__ sgt = A.sig + (size_t)2 * U * A.nlp + lih;
      for (int p = hw; p < NP; p += 2) cp_async4(ssg + p * W + hc, sgt + (size_t)p * A.nlp);
      cp_async_wait_all();
      asm volatile("bar.sync 1, %0;" ::"r"(NS) : "memory");
      if (lane == 0) mbar_arrive(&sigbar);
    }
    // the chunks as the sweeps finish them, the last first: the outward pass (walls) and the
    // cyclic correction (periodic y) both release the positions nearest the middle first
    for (int ci = 0; ci < nchunk - 1; ++ci) {   // (chunk 0: the sweeps)
      const int c = nchunk - 1 - ci;
      const int lo = U * c, n = min(U, R - lo);
      ok &= mbar_wait_idle(&donebar[c], 0);
      // rows h / W + 2 k of the chunk's 2 n: the upper positions lo + r, then the lower R + lo + r;
      // the fast path for every value, the general routine again where a warp met another.  The
      // chunk's shared-memory reads come first, all of them: the compiler cannot tell them apart
      // from the global stores and would otherwise chain each row behind the previous store.
      uint32_t sp = 0;
      double vv[U];
      float sgm[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int r = hw + 2 * k;
        const int p = r < n ? lo + r : R + lo + (r - n);
        const bool in = r < 2 * n;
        vv[k] = in ? sg[p * W + hc] : 0.0;
        if constexpr (F32) sgm[k] = in ? ssg[p * W + hc] : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int r = hw + 2 * k;
        if (r < 2 * n) {
          const int p = r < n ? lo + r : R + lo + (r - n);
          const int j = rowof(p);
          const double v = vv[k];
          if constexpr (F32) {
            const uint32_t o = fsconv_narrow_fast((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v), &sp);
            const float x = __uint_as_float(o) * sgm[k];
            if (mine && j >= 0) tile[rs * j + hc] = x;
            else if (zcol) ssg[p * W + hc] = x;    // the zero mode's column: kept for its mean
          } else {
            if (mine && j >= 0) tile[rs * j + hc] = v;
          }
        }
      }
      if constexpr (F32) {
        if (__any_sync(FULL, sp)) {
#pragma unroll 1
          for (int k = 0; k < U; ++k) {
            const int r = hw + 2 * k;
            if (r < 2 * n) {
              const int p = r < n ? lo + r : R + lo + (r - n);
              const int j = rowof(p);
              const float x = fsconv_narrow(sg[p * W + hc]) * ssg[p * W + hc];
              if (mine && j >= 0) tile[rs * j + hc] = x;
              else if (zcol) ssg[p * W + hc] = x;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  // 5. zero mode: hy-weighted mean of its column, subtracted as it leaves.  FP32 fields: the column
  // narrowed and scaled by the helpers like every other (x = sigma y in FP32), its mean taken in
  // FP32 (a gauge constant, exact to FP32 rounding; the weights only on stretched y); FP64 fields
  // in FP64.
  if (zb && tid < 32) {
    if constexpr (F32) {
      // the helpers left the column's FP32 values where its sigma was staged
      const float* const xs = reinterpret_cast<const float*>(st);
      float part = 0.0f;
      for (int j = lane; j < ny; j += 32) {
        const float x = xs[pos(j) * W];
        part += A.hy_uniform ? x : (float)__ldg(A.hy + j) * x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
      const float zm = part * (A.hy_uniform ? 1.0f / (float)ny : (float)A.hysum_inv);
      for (int j = lane; j < ny; j += 32) tile[rs * j] = xs[pos(j) * W] - zm;
    } else {
      double part = 0.0;
      for (int j = lane; j < ny; j += 32) part = fma(__ldg(A.hy + j), sg[pos(j) * W], part);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
      const T zm = (T)(part * A.hysum_inv);
      for (int j = lane; j < ny; j += 32) tile[rs * j] = sg[pos(j) * W] - zm;
    }
  }
  if (!ok) atomicOr(A.status, 1u);   // part of the tile never arrived: this block's columns are invalid
}

// ---------------------------------------------------------------------------
// Periodic y: the columns (slot s, z position t) of the x/z spectrum are real
// sequences along y to which the real symmetric circulant inverse
// (A_y + Lambda_s)^-1 applies.  Two neighbouring slots (s, s+1) form one complex
// line z = a + i b; after its DFT Z(k) = A(k) + i B(k), the solution spectrum is
//   Z'(k) = A(k) / mu_a(k) + i B(k) / mu_b(k)
//         = Z(k) (1/mu_a + 1/mu_b) / 2 + conj Z(-k) (1/mu_a - 1/mu_b) / 2,
// mu(k) = lambda_y(k) + Lambda (both slots of a pair share Lambda except the
// special slots 0 and 1 of the real-packed x spectrum and DCT slots).  1/mu is
// taken as 0 for the one zero eigenvalue (k = 0 of the x/z zero mode), which
// gives the zero-mean solution.
struct YSpecArgs {
  int nx, ny, nz, dim, xmode, nmx, spb;
};

template <typename T>
__device__ __forceinline__ int lam_index_spec(const YSpecArgs& A, int s, int t) {
  int mx;
  if (A.xmode == 1) mx = s;
  else mx = s == 0 ? 0 : (s == 1 ? A.nx / 2 : (s >> 1));
  if (A.dim == 2) return mx;
  const int l = (s >= 2 || A.xmode == 1) ? t : (t == 0 ? 0 : (t == 1 ? A.nz / 2 : (t >> 1)));
  return min(l, A.nz - l) * A.nmx + mx;
}

template <typename T, int PL, int NT = 256>
__global__ void __launch_bounds__(NT) yspec_kernel(T* __restrict__ data, const YSpecArgs A, Radices rad,
                                                    const cplx<T>* __restrict__ tw, const T* __restrict__ lamy,
                                                    const T* __restrict__ lamxz) {
  extern __shared__ unsigned char smem_raw[];
  // compile-time lengths up to 640 move 32-slot tiles (spb == 32); longer columns (a few lines
  // per block) move their slots with the generic loops
  constexpr bool TILE32 = PL >= 2 && PL <= 640;
  const int N = PL >= 2 ? PL : A.ny;
  const int P = N + 1;                          // padded line pitch
  cplx<T>* B0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* B1 = B0 + (size_t)(A.spb / 2) * P;
  const int s0 = blockIdx.x * A.spb;
  const int t = blockIdx.y;
  const int ns = min(A.spb, A.nx - s0);
  const int nl = (ns + 1) / 2;
  T* base = data + s0 + (size_t)A.nx * A.ny * t;
  const size_t rs = (size_t)A.nx;
  if (ns & 1)   // odd tail: the missing partner slot is zero
    for (int j = threadIdx.x; j < N; j += blockDim.x) B0[(nl - 1) * P + j].y = T(0);
  if constexpr (TILE32) {
    // spb == 32: thread = (slot c, rows j0 + 8 q)
    const int c = threadIdx.x & 31, j0 = threadIdx.x >> 5;
    if (c < ns) {
      constexpr int NQ = PL / 8;
      T v[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] = base[rs * (j0 + 8 * q) + c];
#pragma unroll
      for (int q = 0; q < NQ; ++q) reinterpret_cast<T*>(&B0[(c >> 1) * P + j0 + 8 * q])[c & 1] = v[q];
    }
  } else {
    constexpr int KB = 8;
    for (int e0 = threadIdx.x; e0 < ns * N; e0 += KB * blockDim.x) {
      T v[KB];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int e = e0 + q * blockDim.x;
        if (e < ns * N) {
          const int j = e / ns, c = e - j * ns;
          v[q] = base[rs * j + c];
        }
      }
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int e = e0 + q * blockDim.x;
        if (e < ns * N) {
          const int j = e / ns, c = e - j * ns;
          reinterpret_cast<T*>(&B0[(c >> 1) * P + j])[c & 1] = v[q];
        }
      }
    }
  }
  __syncthreads();
  cplx<T>* Z = fft_any<T, PL>(B0, B1, N, P, nl, rad, tw, false);
  const int nh = N / 2 + 1;
  for (int e = threadIdx.x; e < nl * nh; e += blockDim.x) {
    const int l = e / nh, k = e - l * nh;
    const int kk = k == 0 ? 0 : N - k;
    const int sa = s0 + 2 * l, sb = sa + 1;
    const T La = lamxz[lam_index_spec<T>(A, sa, t)];
    const T Lb = sb < A.nx ? lamxz[lam_index_spec<T>(A, sb, t)] : La;
    const T ly = lamy[k];
    const T ma = ly + La, mb = ly + Lb;
    const T ia = ma != T(0) ? T(1) / ma : T(0);
    const T ib = mb != T(0) ? T(1) / mb : T(0);
    const T cp = T(0.5) * (ia + ib), cm = T(0.5) * (ia - ib);
    cplx<T>* line = Z + l * P;
    const cplx<T> z1 = line[k], z2 = line[kk];
    line[k] = {cp * z1.x + cm * z2.x, cp * z1.y - cm * z2.y};
    if (kk != k) line[kk] = {cp * z2.x + cm * z1.x, cp * z2.y - cm * z1.y};
  }
  __syncthreads();
  cplx<T>* W = fft_any<T, PL>(Z, Z == B0 ? B1 : B0, N, P, nl, rad, tw, true);
  const T inv_n = T(1) / T(N);
  if constexpr (TILE32) {
    const int c = threadIdx.x & 31, j0 = threadIdx.x >> 5;
    if (c < ns) {
#pragma unroll 4
      for (int q = 0; q < PL / 8; ++q) {
        const int j = j0 + 8 * q;
        const cplx<T> v = W[(c >> 1) * P + j];
        base[rs * j + c] = ((c & 1) ? v.y : v.x) * inv_n;
      }
    }
  } else {
    for (int e = threadIdx.x; e < ns * N; e += blockDim.x) {
      const int j = e / ns, c = e - j * ns;
      const cplx<T> v = W[(c >> 1) * P + j];
      base[rs * j + c] = ((c & 1) ? v.y : v.x) * inv_n;
    }
  }
}

#include "fft_reg.cuh"

template <typename T>
size_t fft_smem_bytes(int N, int lines) {
  return 2ull * lines * N * sizeof(cplx<T>);
}

// z transforms use a padded line pitch N + 1
template <typename T>
size_t fft_smem_bytes_z(int N, int lines) {
  return 2ull * lines * (N + 1) * sizeof(cplx<T>);
}

Radices radices_of(const Plan1D& p) {
  Radices r;
  r.nst = p.nst;
  for (int i = 0; i < FS_MAX_RADIX_STAGES; ++i) r.r[i] = i < p.nst ? p.radix[i] : 1;
  return r;
}

constexpr size_t kSmemBudget = 96 * 1024;
constexpr size_t kFixedBudget = 200 * 1024;   // compile-time-length kernels always take kMaxLines lines
constexpr size_t kYSpecBudget = 200 * 1024;

template <typename T, int PL>
void set_smem_attrs_plan() {
  const int zb = (int)(PL >= 2 ? kFixedBudget : kSmemBudget);
  // (x lines are sized against kSmemBudget; a single line longer than that, FP64 rows beyond 3072
  // points, takes up to kFixedBudget)
  cudaFuncSetAttribute(xfwd_kernel<T, PL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFixedBudget);
  cudaFuncSetAttribute(xfwd_kernel<T, PL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFixedBudget);
  cudaFuncSetAttribute(xinv_kernel<T, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFixedBudget);
  cudaFuncSetAttribute(zfwd_kernel<T, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, zb);
  cudaFuncSetAttribute(zinv_kernel<T, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, zb);
  cudaFuncSetAttribute(yspec_kernel<T, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kYSpecBudget);
  if constexpr (PL == 0) {
    cudaFuncSetAttribute(yspec_kernel<T, 0, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kYSpecBudget);
    cudaFuncSetAttribute(xfwd4k_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)x4_smem_bytes<T>());
    cudaFuncSetAttribute(xfwd4k_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)x4_smem_bytes<T>());
    cudaFuncSetAttribute(xinv4k_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)x4_smem_bytes<T>());
    // (FP64 tiles of the 4096-row y solve exceed the 48 KB default)
    cudaFuncSetAttribute(y4_outer_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)y4_smem_bytes<T>());
    cudaFuncSetAttribute(y4_outer_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)y4_smem_bytes<T>());
    cudaFuncSetAttribute(y4_mid_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)y4_smem_bytes<T>());
    cudaFuncSetAttribute(xfwd_kernel<T, 5760, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFixedBudget);
    cudaFuncSetAttribute(xfwd_kernel<T, 5760, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFixedBudget);
    cudaFuncSetAttribute(xinv_kernel<T, 5760>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFixedBudget);
  }
}

// Kernel instances by plan: compile-time lengths first, generic plans otherwise.
template <typename T>
struct FftKernels {
  using XF = void (*)(T*, int, int, int, int, Radices, const cplx<T>*, const cplx<T>*, const DivArgs<T>);
  using XI = void (*)(T*, int, int, int, int, Radices, const cplx<T>*, const cplx<T>*);
  using ZK = void (*)(T*, int, int, int, int, Radices, const cplx<T>*);
  using YK = void (*)(T*, const YSpecArgs, Radices, const cplx<T>*, const T*, const T*);
  XF xfwd, xfwd_div;
  XI xinv;
  ZK zfwd, zinv;
  YK yspec;
};

template <typename T, int PL>
FftKernels<T> fft_kernels_of() {
  return {xfwd_kernel<T, PL, false>, xfwd_kernel<T, PL, true>, xinv_kernel<T, PL>, zfwd_kernel<T, PL>,
          zinv_kernel<T, PL>, yspec_kernel<T, PL>};
}

// Lengths with compile-time plans: the powers of two and the multiples of 32 up to
// 512 met by the benchmark grids, and 640.  The z and periodic-y kernels of a
// compile-time length stage kMaxLines lines of two buffers in shared memory, so
// a length takes its compile-time plan only where those fit (FP64: n <= 399).
template <typename T>
bool is_fixed_length(int n) {
  switch (n) {
    case 64: case 128: case 160: case 192: case 224: case 256: case 288: case 320: case 352: case 384:
    case 416: case 448: case 480: case 512: case 640:
      return 2ull * kMaxLines * (n + 1) * sizeof(cplx<T>) <= kFixedBudget;
    default:
      return false;
  }
}

template <typename T>
FftKernels<T> fft_kernels(const Plan1D& p) {
  if (is_fixed_length<T>(p.n)) {
    switch (p.n) {
      case 64: return fft_kernels_of<T, 64>();
      case 128: return fft_kernels_of<T, 128>();
      case 160: return fft_kernels_of<T, 160>();
      case 192: return fft_kernels_of<T, 192>();
      case 224: return fft_kernels_of<T, 224>();
      case 256: return fft_kernels_of<T, 256>();
      case 288: return fft_kernels_of<T, 288>();
      case 320: return fft_kernels_of<T, 320>();
      case 352: return fft_kernels_of<T, 352>();
      case 384: return fft_kernels_of<T, 384>();
      case 416: return fft_kernels_of<T, 416>();
      case 448: return fft_kernels_of<T, 448>();
      case 480: return fft_kernels_of<T, 480>();
      case 512: return fft_kernels_of<T, 512>();
      case 640: return fft_kernels_of<T, 640>();
      default: break;
    }
  }
  for (int i = 0; i < p.nst; ++i)
    if (p.radix[i] > 5) return fft_kernels_of<T, 1>();
  return fft_kernels_of<T, 0>();
}

// Rows of 5760 points take a compile-time plan in the x transforms (one line per block); the
// 16-line z and y kernels of that length are not built.  Rows of 4096 points have their own
// radix-16 kernels (xfwd4k_kernel, xinv4k_kernel) and periodic-y columns of 4096 points the
// three-launch four-step solve (y4_outer_kernel, y4_mid_kernel).
constexpr int kXLong2 = 5760;   // 2^7 3^2 5: the rows of the 2-D cylinder-array workload
template <typename T, int N>
FftKernels<T> fft_kernels_xlong() {
  FftKernels<T> K = fft_kernels_of<T, 0>();
  K.xfwd = xfwd_kernel<T, N, false>;
  K.xfwd_div = xfwd_kernel<T, N, true>;
  K.xinv = xinv_kernel<T, N>;
  return K;
}
template <typename T>
FftKernels<T> fft_kernels_x(const Plan1D& p) {
  if (p.n == kXLong2) return fft_kernels_xlong<T, kXLong2>();
  return fft_kernels<T>(p);
}

template <typename T, int N>
void set_smem_attrs_reg() {
  const int b = (int)reg_smem_bytes<T, N>(1);
  cudaFuncSetAttribute(xfwd_reg_kernel<T, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  cudaFuncSetAttribute(xfwd_reg_kernel<T, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  cudaFuncSetAttribute(xinv_reg_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  cudaFuncSetAttribute(zfwd_reg_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  cudaFuncSetAttribute(zinv_reg_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  cudaFuncSetAttribute(yspec_reg_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

bool is_reg_length(int n) { return n == 64 || n == 128 || n == 256 || n == 384 || n == 512; }

// Lines per block of the mixed-radix x transforms: up to 16, fewer when the
// grid has too few lines to give every SM two blocks (2-D grids).
int default_lines(int lines) { return std::max(1, std::min(kMaxLines, lines / (2 * 148))); }

// The register x transforms hold kRegLines lines per block; 2-D grids with
// fewer lines than one such block per SM take the mixed-radix kernels, whose
// block size adapts to the line count.
bool x_reg(const fs_grid* G) {
  return is_reg_length(G->nx) && (G->dim == 3 || (G->ny + 1) / 2 >= kRegLines * 148);
}

// Launches of the register-FFT kernels for a length known at compile time.
template <typename T, int N>
struct RegLaunch {
  static void xfwd(fs_grid* G, T* data, int rows, const DivArgs<T>* dv) {
    const int nb = ((rows + 1) / 2 + kRegLines - 1) / kRegLines;
    const DivArgs<T> none{};
    const size_t sm = reg_smem_bytes<T, N>(0);
    if (dv)
      launch_pdl(G, "fft_x_fwd_div", xfwd_reg_kernel<T, N, true>, dim3(nb), dim3(kRegBlock), sm, data, rows, G->xmode,
                 (const cplx<T>*)G->px.tw, (const cplx<T>*)G->px.dtw, *dv);
    else
      launch_pdl(G, "fft_x_fwd", xfwd_reg_kernel<T, N, false>, dim3(nb), dim3(kRegBlock), sm, data, rows, G->xmode,
                 (const cplx<T>*)G->px.tw, (const cplx<T>*)G->px.dtw, none);
  }
  static void xinv(fs_grid* G, T* data, int rows) {
    const int nb = ((rows + 1) / 2 + kRegLines - 1) / kRegLines;
    launch_pdl(G, "fft_x_inv", xinv_reg_kernel<T, N>, dim3(nb), dim3(kRegBlock), reg_smem_bytes<T, N>(0), data, rows,
               G->xmode, (const cplx<T>*)G->px.tw, (const cplx<T>*)G->px.dtw);
  }
  // tiles [tile0, tile0 + ntiles) of kRegLines slot pairs (ntiles <= 0: every tile)
  static void zfwd(fs_grid* G, T* data, int tile0 = 0, int ntiles = 0) {
    const int nt = ntiles > 0 ? ntiles : (G->nx / 2 + kRegLines - 1) / kRegLines;
    launch_pdl(G, "fft_z_fwd", zfwd_reg_kernel<T, N>, dim3(nt, G->ny), dim3(kRegBlock), reg_smem_bytes<T, N>(0), data,
               G->nx, G->ny, (const cplx<T>*)G->pz.tw, tile0);
  }
  static void zinv(fs_grid* G, T* data, int tile0 = 0, int ntiles = 0) {
    const int nt = ntiles > 0 ? ntiles : (G->nx / 2 + kRegLines - 1) / kRegLines;
    launch_pdl(G, "fft_z_inv", zinv_reg_kernel<T, N>, dim3(nt, G->ny), dim3(kRegBlock), reg_smem_bytes<T, N>(1), data,
               G->nx, G->ny, (const cplx<T>*)G->pz.tw, tile0);
  }
  static void yspec(fs_grid* G, T* data, const YSpecArgs& A) {
    const dim3 grid((G->nx + 31) / 32, G->dim == 3 ? G->nz : 1);
    launch_pdl(G, "fft_y_solve", yspec_reg_kernel<T, N>, grid, dim3(kRegBlock), reg_smem_bytes<T, N>(0), data, A,
               (const cplx<T>*)G->py.tw, (const T*)G->lamy, (const T*)G->lamxz);
  }
};

template <typename T, typename F>
void with_reg_length(int n, F&& f) {
  if (n == 64) f(RegLaunch<T, 64>());
  else if (n == 128) f(RegLaunch<T, 128>());
  else if (n == 256) f(RegLaunch<T, 256>());
  else if (n == 384) f(RegLaunch<T, 384>());
  else f(RegLaunch<T, 512>());
}

template <typename T>
void set_smem_attrs() {
  static bool done = false;
  if (done) return;
  set_smem_attrs_reg<T, 64>();
  set_smem_attrs_reg<T, 128>();
  set_smem_attrs_reg<T, 256>();
  set_smem_attrs_reg<T, 384>();
  set_smem_attrs_reg<T, 512>();
  set_smem_attrs_plan<T, 0>();
  set_smem_attrs_plan<T, 1>();
  set_smem_attrs_plan<T, 64>();
  set_smem_attrs_plan<T, 128>();
  set_smem_attrs_plan<T, 160>();
  set_smem_attrs_plan<T, 192>();
  set_smem_attrs_plan<T, 224>();
  set_smem_attrs_plan<T, 256>();
  set_smem_attrs_plan<T, 288>();
  set_smem_attrs_plan<T, 320>();
  set_smem_attrs_plan<T, 352>();
  set_smem_attrs_plan<T, 384>();
  set_smem_attrs_plan<T, 416>();
  set_smem_attrs_plan<T, 448>();
  set_smem_attrs_plan<T, 480>();
  set_smem_attrs_plan<T, 512>();
  set_smem_attrs_plan<T, 640>();
  if constexpr (std::is_same<T, float>::value) {
    cudaFuncSetAttribute(xzfwd_plane_kernel<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem_bytes<128>());
    cudaFuncSetAttribute(xzfwd_plane_kernel<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem_bytes<128>());
    cudaFuncSetAttribute(zxinv_plane_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem_bytes<128>());
    cudaFuncSetAttribute(xzfwd_plane_kernel<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem_bytes<64>());
    cudaFuncSetAttribute(xzfwd_plane_kernel<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem_bytes<64>());
    cudaFuncSetAttribute(zxinv_plane_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem_bytes<64>());
    cudaFuncSetAttribute(xzfwd_pair_kernel<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_pair_smem_bytes<128>());
    cudaFuncSetAttribute(xzfwd_pair_kernel<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_pair_smem_bytes<128>());
    cudaFuncSetAttribute(zxinv_pair_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_pair_smem_bytes<128>());
  }
  cudaFuncSetAttribute(ysolve_kernel<T, 4, YCOLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  cudaFuncSetAttribute(ysolve_kernel<T, 8, YCOLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  cudaFuncSetAttribute(ysolve_kernel<T, 16, YCOLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  cudaFuncSetAttribute(ysolve_kernel<T, 4, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  cudaFuncSetAttribute(ysolve_kernel<T, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  cudaFuncSetAttribute(ysolve_kernel<T, 16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  cudaFuncSetAttribute(ytwist_kernel<T, true, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  cudaFuncSetAttribute(ytwist_kernel<T, false, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  cudaFuncSetAttribute(ytwist_kernel<T, true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  cudaFuncSetAttribute(ytwist_kernel<T, false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  done = true;
}


}  // namespace

size_t ysolve_smem(int ny, int nseg, int yc) {
  const size_t pitch = ny + (ny & 1);
  const size_t staged = yc == 8 ? (size_t)(4 * yc + 1) * (pitch + 2) : 0;
  return ((size_t)ny * yc + (size_t)yc * 3 * nseg + staged) * sizeof(double);
}

// 3-D tensor map of an FP32 spectrum array [nz][ny][nx] with boxes of w slots x kTwBoxRows rows,
// for the twisted y solve's tile loads; false when the driver's encoder is unavailable or rejects it
bool encode_spectrum_map(CUtensorMap* map, const float* data, int nx, int ny, int nz, int w) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode enc = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      enc = reinterpret_cast<Encode>(fn);
  }
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)nx * ny * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)w, (cuuint32_t)kTwBoxRows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(data), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The twisted y solve over column blocks [xblk0, xblk0 + nxblk) along x (nxblk <= 0: all).
template <typename T>
void launch_ytwist(fs_grid* G, T* data, int xblk0, int nxblk) {
  const int nx = G->nx, ny = G->ny, nz = G->nz;
  YTwArgs A;
  A.nx = nx;
  A.ny = ny;
  A.nz = nz;
  A.dim = G->dim;
  A.xmode = G->xmode;
  A.nmx = G->nmx;
  A.nlz = G->nlz;
  A.L = G->ytw_L;
  A.R = G->ytw_R;
  A.nlp = G->ytw_nlp;
  A.M = G->twM;
  A.E = G->twE;
  A.C = G->twC;
  A.sig = G->twSig;
  A.sig0 = G->twSig0;
  A.P = G->twP;
  A.Z = G->twZ;
  A.S = G->twS;
  A.K = G->twK;
  A.hy = G->hy64;
  A.hysum_inv = 1.0 / G->hysum;
  A.hy_uniform = G->yuniform;
  A.gauge = G->ygauge ? 1 : 0;
  A.status = G->dstatus;
  A.xblk0 = xblk0;
  // rows move by bulk copies when every row start and width is a multiple of 16 bytes
  A.bulk = (nx * (int)sizeof(T)) % 16 == 0 && reinterpret_cast<uintptr_t>(data) % 16 == 0;
  const int w = G->ytw_cols;
  // FP32 tiles of at least one box of rows arrive as tensor-map boxes (a few large copies
  // instead of one bulk copy per row); the map is encoded once per spectrum array
  CUtensorMap tmap;
  std::memset(&tmap, 0, sizeof(tmap));
  A.tiled = 0;
  // (odd chains on walls, ny odd, keep the row copies: the lower thread's first slot is then the
  // inert one, and its first chunk no longer covers the bottom box's rows)
  if (sizeof(T) == 4 && A.bulk && ny >= 2 * kTwBoxRows && ny <= 20 * kTwBoxRows && G->tune_ytile &&
      !(!G->cyclic && (ny & 1))) {
    const int nzt = G->dim == 3 ? nz : 1;
    if (G->ytw_map_ptr != (const void*)data || G->ytw_map_w != w) {
      G->ytw_map_ok = encode_spectrum_map(reinterpret_cast<CUtensorMap*>(G->ytw_map), (const float*)data, nx, ny,
                                          nzt, w);
      G->ytw_map_ptr = data;
      G->ytw_map_w = w;
    }
    if (G->ytw_map_ok) {
      std::memcpy(&tmap, G->ytw_map, sizeof(tmap));
      A.tiled = 1;
    }
  }
  const dim3 grid(nxblk > 0 ? nxblk : (nx + w - 1) / w, G->dim == 3 ? nz : 1);
  const size_t sb = ytwist_smem<T>(ny, w);
  if (w == 64) {
    if (G->cyclic) launch_pdl(G, "ysolve", ytwist_kernel<T, true, 64>, grid, dim3(256), sb, data, A, tmap);
    else launch_pdl(G, "ysolve", ytwist_kernel<T, false, 64>, grid, dim3(256), sb, data, A, tmap);
  } else {
    if (G->cyclic) launch_pdl(G, "ysolve", ytwist_kernel<T, true, 32>, grid, dim3(128), sb, data, A, tmap);
    else launch_pdl(G, "ysolve", ytwist_kernel<T, false, 32>, grid, dim3(128), sb, data, A, tmap);
  }
}

// The x and z transforms fused per y position (xzfwd_plane_kernel, zxinv_plane_kernel): FP32
// fields, nx = nz of 64 or 128, periodic x, the divergence formed from row quads.
template <typename T>
bool xz_plane(const fs_grid* G, const DivArgs<T>* dv) {
  if constexpr (!std::is_same<T, float>::value) {
    return false;
  } else {
    return G->tune_xzplane && G->dim == 3 && G->nx == G->nz && (G->nx == 64 || G->nx == 128) && G->xmode == 0 &&
           (!dv || dv->vec4);
  }
}

template <typename T>
void launch_xz_plane(fs_grid* G, T* data, const DivArgs<T>* dv, bool inverse) {
  if constexpr (std::is_same<T, float>::value) {
    const DivArgs<float> none{};
    const cplx<float>* tw = (const cplx<float>*)G->px.tw;
    const dim3 grid(G->ny);
    if (G->tune_xzplane == 2) {   // two-block clusters: grid of 2 ny blocks
      const dim3 g2(2 * G->ny);
      if (G->nx == 128) {
        if (inverse)
          launch_pdl(G, "fft_xz_inv", zxinv_pair_kernel<128>, g2, dim3(256), plane_pair_smem_bytes<128>(), data, G->ny,
                     tw);
        else
          launch_pdl(G, dv ? "fft_xz_fwd_div" : "fft_xz_fwd",
                     dv ? xzfwd_pair_kernel<128, true> : xzfwd_pair_kernel<128, false>, g2, dim3(256),
                     plane_pair_smem_bytes<128>(), data, G->ny, tw, dv ? *dv : none);
      } else {
        if (inverse)
          launch_pdl(G, "fft_xz_inv", zxinv_pair_kernel<64>, g2, dim3(128), plane_pair_smem_bytes<64>(), data, G->ny, tw);
        else
          launch_pdl(G, dv ? "fft_xz_fwd_div" : "fft_xz_fwd",
                     dv ? xzfwd_pair_kernel<64, true> : xzfwd_pair_kernel<64, false>, g2, dim3(128),
                     plane_pair_smem_bytes<64>(), data, G->ny, tw, dv ? *dv : none);
      }
      return;
    }
    if (G->nx == 128) {
      if (inverse)
        launch_pdl(G, "fft_xz_inv", zxinv_plane_kernel<128>, grid, dim3(1024), plane_smem_bytes<128>(), data, G->ny, tw);
      else
        launch_pdl(G, dv ? "fft_xz_fwd_div" : "fft_xz_fwd",
                   dv ? xzfwd_plane_kernel<128, true> : xzfwd_plane_kernel<128, false>, grid, dim3(1024),
                   plane_smem_bytes<128>(), data, G->ny, tw, dv ? *dv : none);
    } else {
      if (inverse)
        launch_pdl(G, "fft_xz_inv", zxinv_plane_kernel<64>, grid, dim3(512), plane_smem_bytes<64>(), data, G->ny, tw);
      else
        launch_pdl(G, dv ? "fft_xz_fwd_div" : "fft_xz_fwd",
                   dv ? xzfwd_plane_kernel<64, true> : xzfwd_plane_kernel<64, false>, grid, dim3(512),
                   plane_smem_bytes<64>(), data, G->ny, tw, dv ? *dv : none);
    }
  }
}

template <typename T>
void poisson_solve(fs_grid* G, T* data, const DivArgs<T>* dv) {
  set_smem_attrs<T>();
  const int nx = G->nx, ny = G->ny, nz = G->nz;
  const int rows = ny * nz;
  // Periodic-z grids with the twisted y solve in two or more column blocks along x: the z
  // transforms and the y solve of the two halves of the x spectrum are independent, so they run as
  // two chains on two streams (fork after the x transform, join before its inverse).  The y solve is
  // bound by the FP64 pipe and the z transforms by memory, so each half's y solve runs beside the
  // other half's transforms; each y-solve half also holds one block per SM instead of two.
  const bool zreg2 = G->dim == 3 && is_reg_length(nz);
  const int wcol = G->ytw_cols;
  const int nxb = (nx + wcol - 1) / wcol;
  const int tiles_per_blk = (wcol / 2) / kRegLines;
  const bool split = G->tune_ysplit && zreg2 && G->ytwist && !G->yspec && G->ystream2 && nxb >= 2 &&
                     nx % wcol == 0 && (wcol / 2) % kRegLines == 0;
  const bool plane = !split && xz_plane<T>(G, dv);
  // x forward (and z forward in the fused form)
  if (plane) {
    launch_xz_plane<T>(G, data, dv, false);
  } else if (x_reg(G)) {
    with_reg_length<T>(nx, [&](auto L) { L.xfwd(G, data, rows, dv); });
  } else if (nx == kX4) {
    const DivArgs<T> none{};
    launch_pdl(G, dv ? "fft_x_fwd_div" : "fft_x_fwd", dv ? xfwd4k_kernel<T, true> : xfwd4k_kernel<T, false>,
               dim3((rows + 1) / 2), dim3(256), x4_smem_bytes<T>(), data, rows, G->xmode, (const cplx<T>*)G->px.tw,
               (const cplx<T>*)G->px.dtw, dv ? *dv : none);
  } else {
    int lpb = (int)(kSmemBudget / fft_smem_bytes<T>(nx, 1));
    const int lines = (rows + 1) / 2;
    const int want = G->tune_fft_lines > 0 ? G->tune_fft_lines : default_lines(lines);
    lpb = lpb > want ? want : (lpb < 1 ? 1 : lpb);
    const int nb = (lines + lpb - 1) / lpb;
    const FftKernels<T> K = fft_kernels_x<T>(G->px);
    auto k = dv ? K.xfwd_div : K.xfwd;
    const DivArgs<T> none{};
    FS_LAUNCH(G, dv ? "fft_x_fwd_div" : "fft_x_fwd",
              k<<<nb, 256, fft_smem_bytes<T>(nx, lpb), G->stream>>>(data, nx, rows, lpb, G->xmode, radices_of(G->px),
                                                                    (const cplx<T>*)G->px.tw,
                                                                    (const cplx<T>*)G->px.dtw, dv ? *dv : none));
  }
  if (split) {
    const int hb = nxb / 2;
    const int nt = (nx / 2) / kRegLines;
    cudaEventRecord(G->yev[0], G->stream);
    cudaStreamWaitEvent(G->ystream2, G->yev[0], 0);
    with_reg_length<T>(nz, [&](auto L) { L.zfwd(G, data, 0, hb * tiles_per_blk); });
    launch_ytwist<T>(G, data, 0, hb);
    with_reg_length<T>(nz, [&](auto L) { L.zinv(G, data, 0, hb * tiles_per_blk); });
    cudaStream_t main = G->stream;
    G->stream = G->ystream2;
    with_reg_length<T>(nz, [&](auto L) { L.zfwd(G, data, hb * tiles_per_blk, nt - hb * tiles_per_blk); });
    launch_ytwist<T>(G, data, hb, nxb - hb);
    with_reg_length<T>(nz, [&](auto L) { L.zinv(G, data, hb * tiles_per_blk, nt - hb * tiles_per_blk); });
    cudaEventRecord(G->yev[1], G->stream);
    G->stream = main;
    cudaStreamWaitEvent(G->stream, G->yev[1], 0);
  } else {
    int ppb = 0;
    const bool zreg = G->dim == 3 && is_reg_length(nz);
    if (plane) {
      // z forward done with the x forward
    } else if (zreg) {
      with_reg_length<T>(nz, [&](auto L) { L.zfwd(G, data); });
    } else if (G->dim == 3) {
      if (is_fixed_length<T>(G->pz.n)) {
        ppb = kMaxLines;   // the compile-time-length z kernels map 32 slots x 8 rows onto 256 threads
      } else {
        ppb = (int)(kSmemBudget / fft_smem_bytes_z<T>(nz, 1));
        const int want = G->tune_fft_lines > 0 ? G->tune_fft_lines : kMaxLines;
        ppb = ppb > want ? want : (ppb < 1 ? 1 : ppb);
        if (ppb > nx / 2) ppb = nx / 2;
      }
      dim3 grid((nx / 2 + ppb - 1) / ppb, ny);
      auto k = fft_kernels<T>(G->pz).zfwd;
      FS_LAUNCH(G, "fft_z_fwd", k<<<grid, 256, fft_smem_bytes_z<T>(nz, ppb), G->stream>>>(data, nx, ny, nz, ppb, radices_of(G->pz),
                                                              (const cplx<T>*)G->pz.tw));
    }
    if (G->yspec && is_reg_length(ny)) {
      YSpecArgs A;
      A.nx = nx;
      A.ny = ny;
      A.nz = nz;
      A.dim = G->dim;
      A.xmode = G->xmode;
      A.nmx = G->nmx;
      A.spb = 32;
      with_reg_length<T>(ny, [&](auto L) { L.yspec(G, data, A); });
    } else if (G->yspec && ny == kY4 * kY4) {
      YSpecArgs A;
      A.nx = nx;
      A.ny = ny;
      A.nz = nz;
      A.dim = G->dim;
      A.xmode = G->xmode;
      A.nmx = G->nmx;
      A.spb = 32;
      const dim3 grid((nx + 31) / 32, kY4 / 2, G->dim == 3 ? nz : 1);
      const cplx<T>* tw = (const cplx<T>*)G->py.tw;
      launch_pdl(G, "fft_y_fwd", y4_outer_kernel<T, false>, grid, dim3(kRegBlock), y4_smem_bytes<T>(), data, nx, tw);
      launch_pdl(G, "fft_y_solve", y4_mid_kernel<T>, grid, dim3(kRegBlock), y4_smem_bytes<T>(), data, A, tw,
                 (const T*)G->lamy, (const T*)G->lamxz);
      launch_pdl(G, "fft_y_inv", y4_outer_kernel<T, true>, grid, dim3(kRegBlock), y4_smem_bytes<T>(), data, nx, tw);
    } else if (G->yspec) {
      YSpecArgs A;
      A.nx = nx;
      A.ny = ny;
      A.nz = nz;
      A.dim = G->dim;
      A.xmode = G->xmode;
      A.nmx = G->nmx;
      // slots per block: an even count whose two ping-pong buffers fit the budget
      const size_t line_bytes = 2ull * (ny + 1) * sizeof(cplx<T>);
      int spb = 2 * (int)std::min<size_t>(kMaxLines, kYSpecBudget / line_bytes);
      if (is_fixed_length<T>(ny)) spb = 2 * kMaxLines;   // compile-time lengths map 32 slots x 8 rows onto 256 threads
      else if (G->tune_fft_lines > 0) spb = std::min(spb, 2 * G->tune_fft_lines);
      A.spb = spb;
      dim3 grid((nx + spb - 1) / spb, G->dim == 3 ? nz : 1);
      auto k = fft_kernels<T>(G->py).yspec;
      // long columns (a few lines per block, one block per SM): 1024 threads instead of 256 keep
      // more butterflies of each stage in flight (radices up to 5)
      int nt = 256;
      if (k == yspec_kernel<T, 0> && spb <= 8) {
        k = yspec_kernel<T, 0, 1024>;
        nt = 1024;
      }
      FS_LAUNCH(G, "fft_y_solve", k<<<grid, nt, (size_t)(spb / 2) * line_bytes, G->stream>>>(
                                      data, A, radices_of(G->py), (const cplx<T>*)G->py.tw, (const T*)G->lamy,
                                      (const T*)G->lamxz));
    } else if (G->ytwist) {
      launch_ytwist<T>(G, data, 0, 0);
    } else {
      YArgs A;
      A.nx = nx;
      A.ny = ny;
      A.nz = nz;
      A.dim = G->dim;
      A.xmode = G->xmode;
      A.nmx = G->nmx;
      A.nlz = G->nlz;
      A.cyclic = G->cyclic;
      A.a = G->ya;
      A.E = G->tE;
      A.CP = G->tCP;
      A.ZV = G->tZV;
      A.WV = G->tWV;
      A.MI = G->tMI;
      A.hy = G->hy64;
      A.hysum = G->hysum;
      A.pitch = G->ypitch;
      A.status = G->dstatus;
      // narrow blocks with staged tables when 32-column blocks would leave SMs idle
      const int tz = G->dim == 3 ? nz : 1;
      const int yc = G->ynarrow ? 8 : YCOLS;
      const dim3 grid((nx + yc - 1) / yc, tz);
      const int ns = G->ynseg;
      const size_t sb = ysolve_smem(ny, ns, yc);
      if (yc == 8) {
        if (ns == 16) FS_LAUNCH(G, "ysolve", ysolve_kernel<T, 16, 8><<<grid, dim3(8, 16), sb, G->stream>>>(data, A));
        else if (ns == 8) FS_LAUNCH(G, "ysolve", ysolve_kernel<T, 8, 8><<<grid, dim3(8, 8), sb, G->stream>>>(data, A));
        else FS_LAUNCH(G, "ysolve", ysolve_kernel<T, 4, 8><<<grid, dim3(8, 4), sb, G->stream>>>(data, A));
      } else if (ns == 16) {
        FS_LAUNCH(G, "ysolve", ysolve_kernel<T, 16, YCOLS><<<grid, dim3(YCOLS, 16), sb, G->stream>>>(data, A));
      } else if (ns == 8) {
        FS_LAUNCH(G, "ysolve", ysolve_kernel<T, 8, YCOLS><<<grid, dim3(YCOLS, 8), sb, G->stream>>>(data, A));
      } else {
        FS_LAUNCH(G, "ysolve", ysolve_kernel<T, 4, YCOLS><<<grid, dim3(YCOLS, 4), sb, G->stream>>>(data, A));
      }
    }
    if (plane) {
      // z inverse done with the x inverse
    } else if (zreg) {
      with_reg_length<T>(nz, [&](auto L) { L.zinv(G, data); });
    } else if (G->dim == 3) {
      dim3 grid((nx / 2 + ppb - 1) / ppb, ny);
      auto k = fft_kernels<T>(G->pz).zinv;
      FS_LAUNCH(G, "fft_z_inv", k<<<grid, 256, fft_smem_bytes_z<T>(nz, ppb), G->stream>>>(data, nx, ny, nz, ppb, radices_of(G->pz),
                                                              (const cplx<T>*)G->pz.tw));
    }
  }
  if (plane) {
    launch_xz_plane<T>(G, data, dv, true);
  } else if (x_reg(G)) {
    with_reg_length<T>(nx, [&](auto L) { L.xinv(G, data, rows); });
  } else if (nx == kX4) {
    launch_pdl(G, "fft_x_inv", xinv4k_kernel<T>, dim3((rows + 1) / 2), dim3(256), x4_smem_bytes<T>(), data, rows,
               G->xmode, (const cplx<T>*)G->px.tw, (const cplx<T>*)G->px.dtw);
  } else {
    int lpb = (int)(kSmemBudget / fft_smem_bytes<T>(nx, 1));
    const int lines = (rows + 1) / 2;
    const int want = G->tune_fft_lines > 0 ? G->tune_fft_lines : default_lines(lines);
    lpb = lpb > want ? want : (lpb < 1 ? 1 : lpb);
    const int nb = (lines + lpb - 1) / lpb;
    auto k = fft_kernels_x<T>(G->px).xinv;
    FS_LAUNCH(G, "fft_x_inv", k<<<nb, 256, fft_smem_bytes<T>(nx, lpb), G->stream>>>(data, nx, rows, lpb, G->xmode, radices_of(G->px),
                                                          (const cplx<T>*)G->px.tw, (const cplx<T>*)G->px.dtw));
  }
}

template <typename T>
void poisson_solve_inplace(fs_grid* G, T* data) {
  poisson_solve<T>(G, data, nullptr);
}

template <typename T>
void poisson_solve_from_velocity(fs_grid* G, const DivArgs<T>& div, T* data) {
  poisson_solve<T>(G, data, &div);
}

template void poisson_solve_inplace<float>(fs_grid*, float*);
template void poisson_solve_inplace<double>(fs_grid*, double*);
template void poisson_solve_from_velocity<float>(fs_grid*, const DivArgs<float>&, float*);
template void poisson_solve_from_velocity<double>(fs_grid*, const DivArgs<double>&, double*);

}  // namespace fs
