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
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
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
//
// Periodic y (cyclic): with xi = x_{ny-1}, rows 0..ny-2 read A'' x' = d' - xi u,
// u the coupling column of x_{ny-1}; so x' = y - xi z with A'' y = d' (the solve
// above) and z = A''^-1 u (tabulated), and row ny-1 gives
//   xi = (d_{ny-1} - S0 y_0 - S1 y_{ny-2}) S2,   S2 = 1 / (b_{ny-1} - S0 z_0 - S1 z_{ny-2}),
// S0, S1 its couplings to x_0 and x_{ny-2}: one more multiply-add per row.
//
// Rows are held in "position" order p(j) = j (j <= k), L + k - j (k < j < L),
// ny - 1 (the bordered row): both threads of a column then sweep the same
// direction (positions ascending while eliminating, descending while
// substituting), so the shared-memory tile and the eigenvalue-major tables
// ([nlam][pitch], position order) are read at fixed offsets from one base, the
// tables a chunk of U rows ahead of their use.  The tile's rows arrive by bulk
// asynchronous copies straight into their positions and leave the same way.
// FP32 fields stay FP32 in shared memory: each thread widens its next chunk of
// the spectrum and narrows its solution with integer field arithmetic
// (fpconv.cuh) inside its sweeps, where those instructions issue while the FP64
// pipe, the kernel's bound (one warp instruction per ~73 cycles per SM
// sub-partition on B300, conversions included), works on the chain.
//
// The singular zero mode pins x_0 = 0 through its tables (E_0 = C_0 = 0,
// M_1 = 0, no coupling to row 0) and is shifted to zero hy-weighted mean (with
// FP32 fields the shift, a constant invisible to the pressure gradient, is
// applied after narrowing).
//
// Block: W columns (16 per warp, lanes 0..15 the upper and 16..31 the lower
// threads); 3-D blocks are ordered so that the z positions t and nz - t, which
// share every eigenvalue, run next to each other.
struct YTwArgs {
  int nx, ny, nz, dim, xmode, nmx, nlz;
  int L, k;              // chain rows 0..L-1; the upper thread owns rows 0..k
  int pitch;             // table row pitch (>= ny, even)
  int bulk;              // rows move by bulk copies (16-byte aligned rows and widths)
  const double* M;       // [nlam][pitch] forward multipliers (negated), position order
  const double* E;       // [nlam][pitch] inverse pivots
  const double* C;       // [nlam][pitch] outward multipliers (negated)
  const double* Z;       // [nlam][pitch] cyclic: z = A''^-1 u
  const double* P;       // [nlam][4] inverse of the middle 2x2 system
  const double* S;       // [nlam][4] cyclic: S0, S1, S2
  const double* hy;      // cell widths (zero-mode mean)
  double hysum;
  unsigned* status;      // device status word (bit 0: a bulk copy wait gave up)
};

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
  return (size_t)ny * w * (sizeof(double) + (sizeof(T) == 4 ? sizeof(T) : 0));
}

template <typename T, bool CYC, int W>
__global__ void __launch_bounds__(2 * W) ytwist_kernel(T* __restrict__ data, const YTwArgs A) {
  constexpr bool F32 = sizeof(T) == 4;
  constexpr int U = 16;                          // rows per chunk (tables fetched a chunk ahead)
  constexpr int NG = 4;                          // tile row groups, each on its own barrier
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char ytw_raw[];
  const int ny = A.ny, L = A.L, k = A.k;
  double* sg = reinterpret_cast<double*>(ytw_raw);   // [ny][W] FP64 eliminated / solved values, position order
  T* st = F32 ? reinterpret_cast<T*>(ytw_raw + (size_t)ny * W * sizeof(double)) : reinterpret_cast<T*>(sg);
  __shared__ uint64_t bar[NG];
  const int tid = threadIdx.x, lane = tid & 31, half = lane >> 4;
  const int cb = (tid >> 5) * 16 + (lane & 15);
  const int s0 = blockIdx.x * W;
  const int ncol = min(W, A.nx - s0);
  int t = 0;
  if (A.dim == 3) {
    const int b = blockIdx.y;
    t = (b & 1) ? A.nz - ((b + 1) >> 1) : (b >> 1);
  }
  const size_t rs = (size_t)A.nx;
  T* tile = data + (size_t)A.nx * ny * t + s0;
  auto pos = [&](int j) { return j <= k ? j : (j < L ? L + k - j : j); };
  const int s = s0 + cb;
  const bool act = cb < ncol;
  const int li = act ? lam_of(A.nx, A.nz, A.dim, A.xmode, A.nmx, s, t) : 0;
  const int P0 = half ? k + 1 : 0;             // first position of this thread
  const int R = half ? L - 1 - k : k + 1;      // positions of this thread's elimination
  const int RW = k + 1;                        // the upper thread's count (>= the lower's): warp-uniform trips
  const size_t tb = (size_t)li * A.pitch + P0;
  const double* __restrict__ Mt = A.M + tb;
  // group of a row: by its offset from the first position of its thread (upper rows 0..k, lower
  // rows from position k + 1; the bordered row last), cut at offsets 17, 33, 49 so that group g
  // holds the chunk the elimination widens g-th
  auto group = [&](int j) {
    const int p = pos(j);
    const int off = p >= L ? RW : (p <= k ? p : p - (k + 1));
    return off < 17 ? 0 : min(NG - 1, (off - 1) >> 4);
  };
  // the first multipliers while the tile is in flight (tables do not depend on the predecessor)
  double mn[U];
#pragma unroll
  for (int q = 0; q < U; ++q) mn[q] = (1 + q < R) ? __ldg(Mt + 1 + q) : 0.0;
  bool ok = true;
  if (A.bulk && tid == 0) {
    for (int g = 0; g < NG; ++g) mbar_init(&bar[g], 1);
    mbar_init_fence();
  }
  __syncthreads();
  pdl_wait();
  const uint32_t rb = (uint32_t)(ncol * sizeof(T));
  if (A.bulk) {
    if (tid < 32) {
      if (lane < NG) {
        // rows of group g: offsets [lo, hi) of the upper (RW rows) and lower (L - RW rows) threads,
        // and the bordered row (offset RW) in the group that holds offset RW
        const int lo = lane == 0 ? 0 : 1 + 16 * lane, hi = lane == NG - 1 ? 1 << 30 : 17 + 16 * lane;
        auto cnt = [&](int n) { return max(0, min(hi, n) - lo); };
        int rows = cnt(RW) + cnt(L - RW);
        if (CYC && RW >= lo && RW < hi) ++rows;
        mbar_expect_tx(&bar[lane], rb * (uint32_t)rows);
      }
      __syncwarp();
      // issue in group order so that the first rows needed land first
      for (int g = 0; g < NG; ++g)
        for (int j = lane; j < ny; j += 32)
          if (group(j) == g) bulk_g2s(st + (size_t)pos(j) * W, tile + rs * j, rb, &bar[g]);
    }
  } else {
#pragma unroll 8
    for (int e = tid; e < ny * W; e += 2 * W) {
      const int j = e / W, c = e - j * W;
      if (c < ncol) st[pos(j) * W + c] = tile[rs * j + c];
    }
    __syncthreads();
  }
  auto wait_group = [&](int g) {
    if (A.bulk) ok &= mbar_wait(&bar[min(g, NG - 1)], 0);
  };
  T* op = st + P0 * W + cb;                    // this thread's column of the tile, from its first position
  double* gp = sg + P0 * W + cb;
  // d at positions i0 .. i0 + U - 1 by the integer fast path (positions past R and inactive columns
  // read as zero); `sp` collects the values outside it
  auto widen_fast = [&](int i0, double (&out)[U], uint32_t& sp) {
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int i = i0 + q;
      if constexpr (F32) {
        const uint32_t u = (act && i < R) ? __float_as_uint(op[i * W]) : 0u;
        uint32_t hi, lo;
        fsconv_widen_fast(u, &hi, &lo, &sp);
        out[q] = __hiloint2double((int)hi, (int)lo);
      } else {
        out[q] = (act && i < R) ? (double)op[i * W] : 0.0;
      }
    }
  };
  auto widen_fix = [&](int i0, double (&out)[U], uint32_t sp) {
    if constexpr (F32) {
      if (__any_sync(FULL, sp)) {
#pragma unroll
        for (int q = 0; q < U; ++q) {
          const int i = i0 + q;
          out[q] = (act && i < R) ? fsconv_widen(op[i * W]) : 0.0;
        }
      }
    }
  };
  // FP64 value v of position i narrowed into the tile by the fast path
  auto narrow_fast = [&](int i, double v, uint32_t& sp) {
    if constexpr (F32) {
      const uint32_t r = fsconv_narrow_fast((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v), &sp);
      if (i >= 0 && i < R) op[i * W] = __uint_as_float(r);
    } else {
      if (i >= 0 && i < R) op[i * W] = v;
    }
  };
  // 1. elimination towards the middle; the next chunk is widened (fast path) and its multipliers
  // fetched while the chain runs, its exceptional values redone after
  wait_group(0);
  double gv = act ? widen<T>(op[0]) : 0.0;
  gp[0] = gv;
  double dn[U];
  {
    uint32_t sp = 0;
    widen_fast(1, dn, sp);
    widen_fix(1, dn, sp);
  }
  int c = 0;
  for (int i0 = 1; i0 < RW; i0 += U, ++c) {
    double mc[U], dc[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      mc[q] = mn[q];
      dc[q] = dn[q];
      mn[q] = (i0 + U + q < R) ? __ldg(Mt + i0 + U + q) : 0.0;
    }
    const bool more = i0 + U < RW;
    if (more) wait_group(c + 1);
    uint32_t sp = 0;
    if (more) widen_fast(i0 + U, dn, sp);
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int i = i0 + q;
      if (i < R) {
        gv = fma(mc[q], gv, dc[q]);
        gp[i * W] = gv;
      }
    }
    if (more) widen_fix(i0 + U, dn, sp);
  }
  // 2. the middle rows k (upper's last position) and k+1 (lower's last)
  const double oth = __shfl_xor_sync(FULL, gv, 16);
  const double gk = half ? oth : gv, hk = half ? gv : oth;
  const double* Pt = A.P + (size_t)li * 4 + 2 * half;
  double xv = fma(__ldg(Pt), gk, __ldg(Pt + 1) * hk);
  gp[(R - 1) * W] = xv;
  // 3. outward substitution, step m at position R - 2 - m (walls: narrowed as they are solved)
  {
    const double* __restrict__ Et = A.E + tb;
    const double* __restrict__ Ct = A.C + tb;
    double en[U], cn[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int i = R - 2 - q;
      en[q] = i >= 0 ? __ldg(Et + i) : 0.0;
      cn[q] = i >= 0 ? __ldg(Ct + i) : 0.0;
    }
    for (int m0 = 0; m0 < RW - 1; m0 += U) {
      double ec[U], cc[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        ec[q] = en[q];
        cc[q] = cn[q];
        const int i = R - 2 - (m0 + U + q);
        en[q] = i >= 0 ? __ldg(Et + i) : 0.0;
        cn[q] = i >= 0 ? __ldg(Ct + i) : 0.0;
      }
      uint32_t sp = 0;
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int i = R - 2 - (m0 + q);
        if (i >= 0) {
          const double eg = ec[q] * gp[i * W];
          xv = fma(cc[q], xv, eg);
          gp[i * W] = xv;
        }
        if constexpr (!CYC && F32) narrow_fast(i, xv, sp);
      }
      if constexpr (!CYC && F32) {
        if (__any_sync(FULL, sp)) {
#pragma unroll
          for (int q = 0; q < U; ++q) {
            const int i = R - 2 - (m0 + q);
            if (i >= 0) op[i * W] = fsconv_narrow(gp[i * W]);
          }
        }
      }
    }
  }
  pdl_trigger();
  if constexpr (CYC) {
    // 4. the bordered row ny - 1 (position ny - 1), then x = y - xi z, narrowed
    for (int g = 1; g < NG; ++g) wait_group(g);   // the bordered row's group (already complete but for short columns)
    const double o2 = __shfl_xor_sync(FULL, xv, 16);
    const double y0 = half ? o2 : xv, yl = half ? xv : o2;   // positions 0 and k + 1
    const double* St = A.S + (size_t)li * 4;
    T* lastp = st + (size_t)(ny - 1) * W + cb;
    const double dl = act ? widen<T>(*lastp) : 0.0;
    const double xi = fma(-__ldg(St + 1), yl, fma(-__ldg(St), y0, dl)) * __ldg(St + 2);
    const double* __restrict__ Zt = A.Z + tb;
    double zn[U];
#pragma unroll
    for (int q = 0; q < U; ++q) zn[q] = q < R ? __ldg(Zt + q) : 0.0;
    for (int i0 = 0; i0 < RW; i0 += U) {
      double zc[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        zc[q] = zn[q];
        zn[q] = i0 + U + q < R ? __ldg(Zt + i0 + U + q) : 0.0;
      }
      uint32_t sp = 0;
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int i = i0 + q;
        narrow_fast(i, fma(-xi, zc[q], i < R ? gp[i * W] : 0.0), sp);
      }
      if constexpr (F32) {
        if (__any_sync(FULL, sp)) {
#pragma unroll
          for (int q = 0; q < U; ++q) {
            const int i = i0 + q;
            if (i < R) op[i * W] = fsconv_narrow(fma(-xi, zc[q], gp[i * W]));
          }
        }
      }
    }
    __syncwarp();
    if (half) *lastp = narrow<T>(xi);
  } else {
    // walls: the middle position, which the outward sweep does not cover
    if constexpr (F32) op[(R - 1) * W] = fsconv_narrow(gp[(R - 1) * W]);
  }
  // 5. zero mode: hy-weighted mean of its column (column 0 of the block holding s = 0, t = 0),
  // subtracted in the field precision
  const bool zb = s0 == 0 && (A.dim == 2 || t == 0);
  __syncthreads();
  if (zb) {
    if (tid < 32) {
      T part = 0;
      for (int j = lane; j < ny; j += 32) part += (T)__ldg(A.hy + j) * st[pos(j) * W];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
      const T zm = part / (T)A.hysum;
      for (int p = lane; p < ny; p += 32) st[p * W] -= zm;
    }
    __syncthreads();
  }
  if (A.bulk) {
    fence_proxy_async_smem();
    __syncthreads();
    if (tid < 32) {
      for (int j = lane; j < ny; j += 32) bulk_s2g(tile + rs * j, st + (size_t)pos(j) * W, rb);
      bulk_s2g_commit();
      bulk_s2g_wait();
    }
  } else {
#pragma unroll 8
    for (int e = tid; e < ny * W; e += 2 * W) {
      const int j = e / W, c2 = e - j * W;
      if (c2 < ncol) tile[rs * j + c2] = st[pos(j) * W + c2];
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

template <typename T, int PL>
__global__ void __launch_bounds__(256) yspec_kernel(T* __restrict__ data, const YSpecArgs A, Radices rad,
                                                    const cplx<T>* __restrict__ tw, const T* __restrict__ lamy,
                                                    const T* __restrict__ lamxz) {
  extern __shared__ unsigned char smem_raw[];
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
  if constexpr (PL >= 2) {
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
  if constexpr (PL >= 2) {
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
  cudaFuncSetAttribute(xfwd_kernel<T, PL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget);
  cudaFuncSetAttribute(xfwd_kernel<T, PL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget);
  cudaFuncSetAttribute(xinv_kernel<T, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget);
  cudaFuncSetAttribute(zfwd_kernel<T, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, zb);
  cudaFuncSetAttribute(zinv_kernel<T, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, zb);
  cudaFuncSetAttribute(yspec_kernel<T, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kYSpecBudget);
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

bool is_reg_length(int n) { return n == 64 || n == 128 || n == 256; }

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
  static void zfwd(fs_grid* G, T* data) {
    const dim3 grid((G->nx / 2 + kRegLines - 1) / kRegLines, G->ny);
    launch_pdl(G, "fft_z_fwd", zfwd_reg_kernel<T, N>, grid, dim3(kRegBlock), reg_smem_bytes<T, N>(0), data, G->nx, G->ny,
               (const cplx<T>*)G->pz.tw);
  }
  static void zinv(fs_grid* G, T* data) {
    const dim3 grid((G->nx / 2 + kRegLines - 1) / kRegLines, G->ny);
    launch_pdl(G, "fft_z_inv", zinv_reg_kernel<T, N>, grid, dim3(kRegBlock), reg_smem_bytes<T, N>(1), data, G->nx, G->ny,
               (const cplx<T>*)G->pz.tw);
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
  else f(RegLaunch<T, 256>());
}

template <typename T>
void set_smem_attrs() {
  static bool done = false;
  if (done) return;
  set_smem_attrs_reg<T, 64>();
  set_smem_attrs_reg<T, 128>();
  set_smem_attrs_reg<T, 256>();
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

template <typename T>
void poisson_solve(fs_grid* G, T* data, const DivArgs<T>* dv) {
  set_smem_attrs<T>();
  const int nx = G->nx, ny = G->ny, nz = G->nz;
  const int rows = ny * nz;
  // x forward
  if (x_reg(G)) {
    with_reg_length<T>(nx, [&](auto L) { L.xfwd(G, data, rows, dv); });
  } else {
    int lpb = (int)(kSmemBudget / fft_smem_bytes<T>(nx, 1));
    const int lines = (rows + 1) / 2;
    const int want = G->tune_fft_lines > 0 ? G->tune_fft_lines : default_lines(lines);
    lpb = lpb > want ? want : (lpb < 1 ? 1 : lpb);
    const int nb = (lines + lpb - 1) / lpb;
    const FftKernels<T> K = fft_kernels<T>(G->px);
    auto k = dv ? K.xfwd_div : K.xfwd;
    const DivArgs<T> none{};
    FS_LAUNCH(G, dv ? "fft_x_fwd_div" : "fft_x_fwd",
              k<<<nb, 256, fft_smem_bytes<T>(nx, lpb), G->stream>>>(data, nx, rows, lpb, G->xmode, radices_of(G->px),
                                                                    (const cplx<T>*)G->px.tw,
                                                                    (const cplx<T>*)G->px.dtw, dv ? *dv : none));
  }
  int ppb = 0;
  const bool zreg = G->dim == 3 && is_reg_length(nz);
  if (zreg) {
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
    FS_LAUNCH(G, "fft_y_solve", k<<<grid, 256, (size_t)(spb / 2) * line_bytes, G->stream>>>(
                                    data, A, radices_of(G->py), (const cplx<T>*)G->py.tw, (const T*)G->lamy,
                                    (const T*)G->lamxz));
  } else if (G->ytwist) {
    YTwArgs A;
    A.nx = nx;
    A.ny = ny;
    A.nz = nz;
    A.dim = G->dim;
    A.xmode = G->xmode;
    A.nmx = G->nmx;
    A.nlz = G->nlz;
    A.L = G->ytw_L;
    A.k = G->ytw_k;
    A.pitch = G->ytw_pitch;
    A.M = G->twM;
    A.E = G->twE;
    A.C = G->twC;
    A.P = G->twP;
    A.Z = G->twZ;
    A.S = G->twS;
    A.hy = G->hy64;
    A.hysum = G->hysum;
    A.status = G->dstatus;
    // rows move by bulk copies when every row start and width is a multiple of 16 bytes
    A.bulk = (nx * (int)sizeof(T)) % 16 == 0 && reinterpret_cast<uintptr_t>(data) % 16 == 0;
    const int w = G->ytw_cols;
    const dim3 grid((nx + w - 1) / w, G->dim == 3 ? nz : 1);
    const size_t sb = ytwist_smem<T>(ny, w);
    if (w == 64) {
      if (G->cyclic) launch_pdl(G, "ysolve", ytwist_kernel<T, true, 64>, grid, dim3(128), sb, data, A);
      else launch_pdl(G, "ysolve", ytwist_kernel<T, false, 64>, grid, dim3(128), sb, data, A);
    } else {
      if (G->cyclic) launch_pdl(G, "ysolve", ytwist_kernel<T, true, 32>, grid, dim3(64), sb, data, A);
      else launch_pdl(G, "ysolve", ytwist_kernel<T, false, 32>, grid, dim3(64), sb, data, A);
    }
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
  if (zreg) {
    with_reg_length<T>(nz, [&](auto L) { L.zinv(G, data); });
  } else if (G->dim == 3) {
    dim3 grid((nx / 2 + ppb - 1) / ppb, ny);
    auto k = fft_kernels<T>(G->pz).zinv;
    FS_LAUNCH(G, "fft_z_inv", k<<<grid, 256, fft_smem_bytes_z<T>(nz, ppb), G->stream>>>(data, nx, ny, nz, ppb, radices_of(G->pz),
                                                            (const cplx<T>*)G->pz.tw));
  }
  if (x_reg(G)) {
    with_reg_length<T>(nx, [&](auto L) { L.xinv(G, data, rows); });
  } else {
    int lpb = (int)(kSmemBudget / fft_smem_bytes<T>(nx, 1));
    const int lines = (rows + 1) / 2;
    const int want = G->tune_fft_lines > 0 ? G->tune_fft_lines : default_lines(lines);
    lpb = lpb > want ? want : (lpb < 1 ? 1 : lpb);
    const int nb = (lines + lpb - 1) / lpb;
    auto k = fft_kernels<T>(G->px).xinv;
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
