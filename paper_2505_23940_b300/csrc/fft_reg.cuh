// Register-resident FFT kernels for the transform lengths 64, 128, 256, 384 and 512,
// the x and z transforms fused per y position (nx = nz of 64 or 128), and the
// 4096-point transforms (periodic y in three launches, x rows by radix-16 passes)
// (included by poisson.cu inside its anonymous namespace; uses cplx, cmul,
// DivArgs, div_at, div4_at, YSpecArgs and lam_index_spec from there).
//
// A line of N = R1 * TPL complex values is transformed by TPL threads in two
// passes with one warp-level exchange through shared memory (the four-step
// decomposition n = t + TPL m, k = q + R1 s):
//   pass 1: thread t takes x[t + TPL m], m < R1, forms the R1-point DFT over m
//           and multiplies entry q by W_N^{t q};
//   pass 2: for each q, the TPL-point DFT over t gives X[q + R1 s], s < TPL.
// The small DFTs (4, 8, 16, 32 points) are straight-line code with constant
// twiddles; the 48-point first pass of N = 384 is three 16-point DFTs and
// sixteen 3-point DFTs, its twiddles read from the line's table.  Lines live in shared memory with one pad element every R1 entries
// so that both passes are free of bank conflicts.  Each block holds kRegLines
// lines; kRegLines * TPL of its threads run the transform (a line never spans
// two warps, so the exchange needs only __syncwarp) and all kRegBlock threads
// move data, as whole slot pairs or row vectors, so that more loads are in
// flight than the transform threads alone could issue.
#pragma once

template <int N>
struct RegPlan;
template <>
struct RegPlan<64> {
  static constexpr int R1 = 8, TPL = 8;
};
template <>
struct RegPlan<128> {
  static constexpr int R1 = 16, TPL = 8;
};
template <>
struct RegPlan<256> {
  static constexpr int R1 = 16, TPL = 16;
};
template <>
struct RegPlan<384> {
  static constexpr int R1 = 48, TPL = 8;    // pass 2: six 8-point DFTs per thread
};
template <>
struct RegPlan<512> {
  static constexpr int R1 = 32, TPL = 16;   // pass 2: two 16-point DFTs per thread
};

constexpr int kRegLines = 16;
constexpr int kRegBlock = 256;
// the 384- and 512-point kernels are held to two blocks per SM (at most 128 registers), the
// shorter ones to four (64 registers: 512 blocks of a 128^3 transform in one wave of 148 x 4)
template <int N>
constexpr int kRegMinBlocks = N >= 384 ? 2 : 4;
// the inverse x transform (real-packed or DCT output: more live values) of 256 points: three
template <int N>
constexpr int kRegMinBlocksXinv = N >= 384 ? 2 : (N >= 256 ? 3 : 4);

// Line pitch: the padded length plus one, so that the 16 lines of a block start
// in 16 different bank pairs (2 * pitch = 2 mod 32 words up to a multiple of 16):
// slot-pair tiles (line = slot / 2) are then written and read without conflicts.
template <int N>
__host__ __device__ constexpr int rpitch() {
  return N + N / RegPlan<N>::R1 + 1;
}
template <int N>
__device__ __forceinline__ int rpad(int i) {
  return i + i / RegPlan<N>::R1;
}
// Line s of a 16-line block tile.  With FP32 entries and 8 threads per line (64, 128 and 384
// points) a warp transforms four lines at once, and the plain pitch (9 mod 16 bank pairs) put their
// starts on the in-line stride of 9, so the passes replayed up to three times: those tiles start
// line s at regpitch s + 8 (s mod 2) + s / 2, which keeps the 16 lines of a tile in 16 different
// bank pairs and starts the four lines of a warp 8 bank pairs apart.  With 16 threads per line, or
// 16-byte FP64 entries, the plain pitch is already conflict-free.
template <typename T, int N>
__host__ __device__ constexpr bool reg_skewed() {
  return sizeof(T) == 4 && RegPlan<N>::TPL == 8;
}
template <typename T, int N>
__host__ __device__ constexpr int regpitch() {
  return reg_skewed<T, N>() ? (N + N / RegPlan<N>::R1 + 23 + 15) / 16 * 16 : rpitch<N>();
}
template <typename T, int N>
__device__ __forceinline__ int regline(int s) {
  if constexpr (reg_skewed<T, N>()) return regpitch<T, N>() * s + 8 * (s & 1) + (s >> 1);
  return rpitch<N>() * s;
}
template <int N>
constexpr int reg_threads() {
  return kRegLines * RegPlan<N>::TPL;
}

template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) {
  return {a.x - b.x, a.y - b.y};
}
// a * (-i) for the forward transform, a * (+i) for the inverse
template <typename T, bool INV>
__device__ __forceinline__ cplx<T> mul_mi(cplx<T> a) {
  return INV ? cplx<T>{-a.y, a.x} : cplx<T>{a.y, -a.x};
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(cplx<T>& a0, cplx<T>& a1, cplx<T>& a2, cplx<T>& a3) {
  const cplx<T> s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const cplx<T> s13 = cadd(a1, a3), d13 = mul_mi<T, INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

// cos and sin of pi/8 and pi/4
constexpr double kC8 = 0.92387953251128675613, kS8 = 0.38268343236508977173, kR2 = 0.70710678118654752440;

// exp(-+ 2 pi i e / 16) for the products e = n2 k1 of the 16-point DFT
template <typename T, bool INV>
__device__ __forceinline__ cplx<T> w16(int e) {
  const T sg = INV ? T(1) : T(-1);
  switch (e) {
    case 1: return {T(kC8), sg * T(kS8)};
    case 2: return {T(kR2), sg * T(kR2)};
    case 3: return {T(kS8), sg * T(kC8)};
    case 4: return {T(0), sg};
    case 6: return {T(-kR2), sg * T(kR2)};
    case 9: return {T(-kC8), -sg * T(kS8)};
    default: return {T(1), T(0)};
  }
}

template <typename T, bool INV>
__device__ __forceinline__ void dft8(cplx<T>* v) {
  cplx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  cplx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<T, INV>(e0, e1, e2, e3);
  dft4<T, INV>(o0, o1, o2, o3);
  const T c = T(kR2), sg = INV ? T(1) : T(-1);
  const cplx<T> t1 = cmul(o1, cplx<T>{c, sg * c});
  const cplx<T> t2 = mul_mi<T, INV>(o2);
  const cplx<T> t3 = cmul(o3, cplx<T>{-c, sg * c});
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1);
  v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2);
  v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3);
  v[7] = csub(e3, t3);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft16(cplx<T>* v) {
  cplx<T> a[4][4];   // a[n2][k1]
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    a[n2][0] = v[n2];
    a[n2][1] = v[4 + n2];
    a[n2][2] = v[8 + n2];
    a[n2][3] = v[12 + n2];
    dft4<T, INV>(a[n2][0], a[n2][1], a[n2][2], a[n2][3]);
  }
#pragma unroll
  for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) a[n2][k1] = cmul(a[n2][k1], w16<T, INV>(n2 * k1));
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cplx<T> c0 = a[0][k1], c1 = a[1][k1], c2 = a[2][k1], c3 = a[3][k1];
    dft4<T, INV>(c0, c1, c2, c3);
    v[k1] = c0;
    v[k1 + 4] = c1;
    v[k1 + 8] = c2;
    v[k1 + 12] = c3;
  }
}

// cos and sin of pi/16 and 3 pi/16
constexpr double kC16 = 0.98078528040323044913, kS16 = 0.19509032201612826785;
constexpr double kC316 = 0.83146961230254523708, kS316 = 0.55557023301960222474;

// exp(-+ 2 pi i k / 32), k < 16
template <typename T, bool INV>
__device__ __forceinline__ cplx<T> w32(int k) {
  const T sg = INV ? T(1) : T(-1);
  const double c[16] = {1.0,  kC16,   kC8,  kC316,  kR2,  kS316,  kS8,  kS16,
                        0.0, -kS16, -kS8, -kS316, -kR2, -kC316, -kC8, -kC16};
  const double s[16] = {0.0, kS16, kS8, kS316, kR2, kC316, kC8, kC16,
                        1.0, kC16, kC8, kC316, kR2, kS316, kS8, kS16};
  return {T(c[k]), sg * T(s[k])};
}

// 32 points: the 16-point DFTs of the even and odd entries, combined (radix 2)
template <typename T, bool INV>
__device__ __forceinline__ void dft32(cplx<T>* v) {
  cplx<T> e[16], o[16];
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    e[n] = v[2 * n];
    o[n] = v[2 * n + 1];
  }
  dft16<T, INV>(e);
  dft16<T, INV>(o);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const cplx<T> t = k == 0 ? o[0] : cmul(o[k], w32<T, INV>(k));
    v[k] = cadd(e[k], t);
    v[k + 16] = csub(e[k], t);
  }
}

// 3 points: y0 = a0 + a1 + a2, y1,2 = a0 - (a1 + a2) / 2 -+ i sqrt(3)/2 (a1 - a2) (forward)
constexpr double kR3h = 0.86602540378443864676;   // sqrt(3) / 2
template <typename T, bool INV>
__device__ __forceinline__ void dft3(cplx<T>& a0, cplx<T>& a1, cplx<T>& a2) {
  const cplx<T> s = cadd(a1, a2), d = csub(a1, a2);
  const cplx<T> t = {a0.x - T(0.5) * s.x, a0.y - T(0.5) * s.y};
  const cplx<T> m0 = mul_mi<T, INV>(d);
  const cplx<T> m = {T(kR3h) * m0.x, T(kR3h) * m0.y};
  a0 = cadd(a0, s);
  a1 = cadd(t, m);
  a2 = csub(t, m);
}

// 48 points (n = 3 n1 + n2, k = k1 + 16 k2): 16-point DFTs over n1, twiddles W_48^{n2 k1}
// (entries st * n2 * k1 of the line's table, st = N / 48), 3-point DFTs over n2
template <typename T, bool INV>
__device__ __forceinline__ void dft48(cplx<T>* v, const cplx<T>* __restrict__ tws, int st) {
  cplx<T> a[3][16];
#pragma unroll
  for (int n2 = 0; n2 < 3; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) a[n2][n1] = v[3 * n1 + n2];
    dft16<T, INV>(a[n2]);
  }
#pragma unroll
  for (int n2 = 1; n2 < 3; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
      cplx<T> w = tws[st * n2 * k1];
      if (INV) w.y = -w.y;
      a[n2][k1] = cmul(a[n2][k1], w);
    }
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) {
    dft3<T, INV>(a[0][k1], a[1][k1], a[2][k1]);
    v[k1] = a[0][k1];
    v[k1 + 16] = a[1][k1];
    v[k1 + 32] = a[2][k1];
  }
}

template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_small(cplx<T>* v) {
  if constexpr (R == 8) dft8<T, INV>(v);
  else if constexpr (R == 16) dft16<T, INV>(v);
  else dft32<T, INV>(v);
}

// Transform the line L (padded layout) in place with the TPL threads t of its
// group; tws holds exp(-2 pi i e / N), e < N.  Every thread of the warp calls it.
template <typename T, int N, bool INV>
__device__ __forceinline__ void fft_reg_line(cplx<T>* L, int t, const cplx<T>* __restrict__ tws) {
  constexpr int R1 = RegPlan<N>::R1, TPL = RegPlan<N>::TPL, G = R1 / TPL;
  cplx<T> v[R1];
#pragma unroll
  for (int m = 0; m < R1; ++m) v[m] = L[rpad<N>(t + TPL * m)];
  if constexpr (R1 == 48) dft48<T, INV>(v, tws, N / 48);
  else dft_small<T, R1, INV>(v);
#pragma unroll
  for (int q = 1; q < R1; ++q) {
    cplx<T> w = tws[t * q];
    if (INV) w.y = -w.y;
    v[q] = cmul(v[q], w);
  }
#pragma unroll
  for (int q = 0; q < R1; ++q) L[rpad<N>(t + TPL * q)] = v[q];
  __syncwarp();
  cplx<T> u[G][TPL];
#pragma unroll
  for (int c = 0; c < G; ++c)
#pragma unroll
    for (int tt = 0; tt < TPL; ++tt) u[c][tt] = L[rpad<N>(tt + TPL * (t * G + c))];
  __syncwarp();
#pragma unroll
  for (int c = 0; c < G; ++c) {
    dft_small<T, TPL, INV>(u[c]);
#pragma unroll
    for (int s = 0; s < TPL; ++s) L[rpad<N>(t * G + c + R1 * s)] = u[c][s];
  }
}

template <typename T, int N>
__device__ __forceinline__ void load_twiddles(cplx<T>* tws, const cplx<T>* __restrict__ tw) {
  for (int e = threadIdx.x; e < N; e += blockDim.x) tws[e] = tw[e];
}

template <typename T, int N>
size_t reg_smem_bytes(int extra_lines) {
  return (size_t)((kRegLines + extra_lines) * regpitch<T, N>() + N) * sizeof(cplx<T>);
}

// The transform threads of the block run the line FFT of their line.
template <typename T, int N, bool INV>
__device__ __forceinline__ void fft_reg_block(cplx<T>* S, const cplx<T>* __restrict__ tws) {
  constexpr int TPL = RegPlan<N>::TPL;
  if (threadIdx.x < reg_threads<N>())
    fft_reg_line<T, N, INV>(S + regline<T, N>(threadIdx.x / TPL), threadIdx.x % TPL, tws);
}

template <typename T>
struct Pair2;
template <>
struct Pair2<float> {
  using V = float2;
};
template <>
struct Pair2<double> {
  using V = double2;
};

// Tile of 32 consecutive slots x N rows (row stride rs) <-> the 16 lines of S:
// slot pair (2m, 2m + 1) is line m (.x, .y).  Thread = (pair m, rows r0 + 16 q);
// pairs are read and written as one 8- (16-) byte vector.  nslots may be odd
// (the missing partner reads as zero and is not written).
template <typename T, int N>
__device__ __forceinline__ void load_pair_tile(cplx<T>* S, const T* __restrict__ base, size_t rs, int nslots) {
  constexpr int NQ = N / 16;
  const int m = threadIdx.x & 15, r0 = threadIdx.x >> 4;
  if (2 * m >= nslots) return;
  const bool whole = 2 * m + 1 < nslots;
  using V = typename Pair2<T>::V;
  cplx<T> v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const T* a = base + rs * (r0 + 16 * q) + 2 * m;
    if (whole) {
      const V w = *reinterpret_cast<const V*>(a);
      v[q] = {w.x, w.y};
    } else {
      v[q] = {a[0], T(0)};
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) S[regline<T, N>(m) + rpad<N>(r0 + 16 * q)] = v[q];
}

template <typename T, int N, typename F>
__device__ __forceinline__ void store_pair_tile(T* __restrict__ base, size_t rs, int nslots, F&& value) {
  constexpr int NQ = N / 16;
  const int m = threadIdx.x & 15, r0 = threadIdx.x >> 4;
  if (2 * m >= nslots) return;
  const bool whole = 2 * m + 1 < nslots;
  using V = typename Pair2<T>::V;
#pragma unroll 4
  for (int q = 0; q < NQ; ++q) {
    const int r = r0 + 16 * q;
    const cplx<T> o = value(m, r);
    T* a = base + rs * r + 2 * m;
    if (whole) {
      V w;
      w.x = o.x;
      w.y = o.y;
      *reinterpret_cast<V*>(a) = w;
    } else {
      a[0] = o.x;
    }
  }
}

// ---------------------------------------------------------------------------
// x forward (see xfwd_kernel): rows of length N, two rows per complex line.
template <typename T, int N, bool DIV>
__global__ void __launch_bounds__(kRegBlock, kRegMinBlocks<N>) xfwd_reg_kernel(T* __restrict__ data, int rows, int mode,
                                                           const cplx<T>* __restrict__ tw,
                                                           const cplx<T>* __restrict__ dtw, const DivArgs<T> dv) {
  pdl_wait();
  constexpr int P = regpitch<T, N>();
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* S = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tws = S + kRegLines * P;
  __shared__ int rowj[2 * kRegLines], rowk[2 * kRegLines];
  const int line0 = blockIdx.x * kRegLines;
  const int nl = min(kRegLines, (rows + 1) / 2 - line0);
  load_twiddles<T, N>(tws, tw);
  if constexpr (DIV) {
    if (threadIdx.x < 2 * nl) {
      const int r = 2 * line0 + threadIdx.x;
      rowk[threadIdx.x] = r / dv.g.ny;
      rowj[threadIdx.x] = r - rowk[threadIdx.x] * dv.g.ny;
    }
    __syncthreads();
  }
  bool done = false;
  if constexpr (DIV) {
    if (dv.vec4 && mode == 0) {
      constexpr int NQ = N / 4;
      constexpr int PER = kRegLines * NQ / kRegBlock;   // quads per thread
      if constexpr (N >= 384 && sizeof(T) == 4) {
        // two blocks per SM (128 registers): the raw loads of two quads of both rows of a line
        // are issued together before any arithmetic (the divergence as div4_at forms it; FP64
        // rows keep the one-quad form, whose registers hold without spilling)
        constexpr int BT = 2;
        static_assert(PER % BT == 0, "whole batches");
        const Geom<T>& g = dv.g;
        const bool d3 = g.dim == 3;
        const int ey = g.ext(1, 1);
        const size_t pu = (size_t)N * g.ny, pv = (size_t)N * ey;
#pragma unroll
        for (int u0 = 0; u0 < PER; u0 += BT) {
          Vec4<T> x[BT][2][5];   // row a, b of the line: u, v at j and j + 1, w at k and k + 1
          T xe[BT][2];           // u right of the quad
#pragma unroll
          for (int b = 0; b < BT; ++b) {
            const int Q = threadIdx.x + kRegBlock * (u0 + b);
            const int l = min(Q / NQ, nl - 1);   // past the block's lines: line nl - 1 again, not stored
            const int i0 = 4 * (Q % NQ);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const bool in = h == 0 || 2 * (line0 + l) + 1 < rows;
              const int j = rowj[2 * l + (in ? h : 0)], k = rowk[2 * l + (in ? h : 0)];
              const T* ur = dv.u[0] + (size_t)N * j + pu * k;
              x[b][h][0] = ld4(ur + i0);
              xe[b][h] = __ldg(ur + (i0 + 4 < N ? i0 + 4 : 0));
              const int jp = j + 1 < ey ? j + 1 : 0;
              const T* vr = dv.u[1] + pv * k + i0;
              x[b][h][1] = ld4(vr + (size_t)N * j);
              x[b][h][2] = ld4(vr + (size_t)N * jp);
              if (d3) {
                const int kp = k + 1 < g.nz ? k + 1 : 0;
                const T* wr = dv.u[2] + (size_t)N * j + i0;
                x[b][h][3] = ld4(wr + pu * k);
                x[b][h][4] = ld4(wr + pu * kp);
              }
            }
          }
#pragma unroll
          for (int b = 0; b < BT; ++b) {
            const int Q = threadIdx.x + kRegBlock * (u0 + b);
            const int l = Q / NQ, i0 = 4 * (Q % NQ);
            if (l < nl) {
              T d[2][4];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const bool in = h == 0 || 2 * (line0 + l) + 1 < rows;
                const T ih = g.ihy[rowj[2 * l + (in ? h : 0)]];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  T sv = ((c < 3 ? x[b][h][0].v[c + 1] : xe[b][h]) - x[b][h][0].v[c]) * g.ihx;
                  sv += (x[b][h][2].v[c] - x[b][h][1].v[c]) * ih;
                  if (d3) sv += (x[b][h][4].v[c] - x[b][h][3].v[c]) * g.ihz;
                  d[h][c] = in ? sv : T(0);
                }
              }
#pragma unroll
              for (int c = 0; c < 4; ++c) S[regline<T, N>(l) + rpad<N>(i0 + c)] = {d[0][c], d[1][c]};
            }
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int Q = threadIdx.x + kRegBlock * u;
          const int l = Q / NQ, i0 = 4 * (Q - l * NQ);
          if (l < nl) {
            const Vec4<T> da = div4_at(dv, i0, rowj[2 * l], rowk[2 * l]);
            Vec4<T> db = {{T(0), T(0), T(0), T(0)}};
            if (2 * (line0 + l) + 1 < rows) db = div4_at(dv, i0, rowj[2 * l + 1], rowk[2 * l + 1]);
#pragma unroll
            for (int e = 0; e < 4; ++e) S[regline<T, N>(l) + rpad<N>(i0 + e)] = {da.v[e], db.v[e]};
          }
        }
      }
      done = true;
    }
  }
  if (!done) {
    constexpr int KB = kRegLines * N / kRegBlock;
    T va[KB], vb[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int t = threadIdx.x + q * kRegBlock;
      const int l = t / N, i = t - l * N;
      va[q] = vb[q] = T(0);
      if (l < nl) {
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
      const int t = threadIdx.x + q * kRegBlock;
      const int l = t / N, i = t - l * N;
      const int dst = mode == 1 ? ((i & 1) ? N - 1 - (i >> 1) : (i >> 1)) : i;
      S[regline<T, N>(l) + rpad<N>(dst)] = {va[q], vb[q]};
    }
  }
  __syncthreads();
  fft_reg_block<T, N, false>(S, tws);
  __syncthreads();
  pdl_trigger();
  // real-packed (periodic) or DCT-II rows; two consecutive outputs per thread
  constexpr int NH = N / 2;
  for (int t = threadIdx.x; t < nl * NH; t += kRegBlock) {
    const int l = t / NH, s0 = 2 * (t - l * NH);
    const int r0 = 2 * (line0 + l), r1 = r0 + 1;
    T oa[2], ob[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int s = s0 + h;
      int m;
      bool im = false;
      if (mode == 0) {
        m = s == 0 ? 0 : (s == 1 ? N / 2 : s >> 1);
        im = s >= 2 && (s & 1);
      } else {
        m = s;
      }
      const cplx<T> z = S[regline<T, N>(l) + rpad<N>(m)], zr = S[regline<T, N>(l) + rpad<N>(m == 0 ? 0 : N - m)];
      const cplx<T> xa = {T(0.5) * (z.x + zr.x), T(0.5) * (z.y - zr.y)};
      const cplx<T> xb = {T(0.5) * (z.y + zr.y), T(0.5) * (zr.x - z.x)};
      if (mode == 0) {
        oa[h] = im ? xa.y : xa.x;
        ob[h] = im ? xb.y : xb.x;
      } else {
        const cplx<T> w = dtw[m];
        oa[h] = w.x * xa.x - w.y * xa.y;
        ob[h] = w.x * xb.x - w.y * xb.y;
      }
    }
    using V = typename Pair2<T>::V;
    V wa, wb;
    wa.x = oa[0];
    wa.y = oa[1];
    wb.x = ob[0];
    wb.y = ob[1];
    *reinterpret_cast<V*>(data + (size_t)r0 * N + s0) = wa;
    if (r1 < rows) *reinterpret_cast<V*>(data + (size_t)r1 * N + s0) = wb;
  }
}

// x inverse (see xinv_kernel)
template <typename T, int N>
__global__ void __launch_bounds__(kRegBlock, kRegMinBlocksXinv<N>) xinv_reg_kernel(T* __restrict__ data, int rows, int mode,
                                                           const cplx<T>* __restrict__ tw,
                                                           const cplx<T>* __restrict__ dtw) {
  pdl_wait();
  constexpr int P = regpitch<T, N>();
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* S = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tws = S + kRegLines * P;
  const int line0 = blockIdx.x * kRegLines;
  const int nl = min(kRegLines, (rows + 1) / 2 - line0);
  load_twiddles<T, N>(tws, tw);
  using V = typename Pair2<T>::V;
  constexpr int KB = kRegLines * N / kRegBlock;
  // entries per thread converted together: all of them up to 256 points; chunks of 8 for the
  // 384- and 512-point rows, whose 24 or 32 pairs of both rows would not fit 128 registers
  constexpr int CH = N >= 384 ? 8 : KB;
  static_assert(KB % CH == 0, "whole chunks");
#pragma unroll
  for (int q0 = 0; q0 < KB; q0 += CH) {
  cplx<T> z[CH];
  if (mode == 0) {
    // Hermitian spectra from real-packed rows: slot pair (2k', 2k' + 1) read as one vector
    V pa[CH], pb[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int t = threadIdx.x + (q0 + q) * kRegBlock;
      const int l = t / N, k = t - l * N;
      const int kk = 2 * k <= N ? k : N - k;
      pa[q].x = pa[q].y = pb[q].x = pb[q].y = T(0);
      if (l < nl) {
        const int r0 = 2 * (line0 + l), r1 = r0 + 1;
        pa[q] = *reinterpret_cast<const V*>(data + (size_t)r0 * N + 2 * (2 * kk == N ? 0 : kk));
        if (r1 < rows) pb[q] = *reinterpret_cast<const V*>(data + (size_t)r1 * N + 2 * (2 * kk == N ? 0 : kk));
      }
    }
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int t = threadIdx.x + (q0 + q) * kRegBlock;
      const int k = t - (t / N) * N;
      cplx<T> xa, xb;
      if (k == 0) {
        xa = {pa[q].x, T(0)};
        xb = {pb[q].x, T(0)};
      } else if (2 * k == N) {
        xa = {pa[q].y, T(0)};
        xb = {pb[q].y, T(0)};
      } else if (2 * k < N) {
        xa = {pa[q].x, pa[q].y};
        xb = {pb[q].x, pb[q].y};
      } else {
        xa = {pa[q].x, -pa[q].y};
        xb = {pb[q].x, -pb[q].y};
      }
      z[q] = {xa.x - xb.y, xa.y + xb.x};   // XA + i XB
    }
  } else {
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int t = threadIdx.x + (q0 + q) * kRegBlock;
      const int l = t / N, k = t - l * N;
      z[q] = {T(0), T(0)};
      if (l < nl) {
        const int r0 = 2 * (line0 + l), r1 = r0 + 1;
        const T* ra = data + (size_t)r0 * N;
        const T* rb = data + (size_t)r1 * N;
        // V[k] = exp(i pi k / 2N) (X[k] - i X[N-k]), X[N] = 0
        const cplx<T> w = cconj(dtw[k]);
        const T a1 = ra[k], a2 = k ? ra[N - k] : T(0);
        const T b1 = r1 < rows ? rb[k] : T(0), b2 = (r1 < rows && k) ? rb[N - k] : T(0);
        const cplx<T> xa = cmul(w, cplx<T>{a1, -a2});
        const cplx<T> xb = cmul(w, cplx<T>{b1, -b2});
        z[q] = {xa.x - xb.y, xa.y + xb.x};
      }
    }
  }
#pragma unroll
  for (int q = 0; q < CH; ++q) {
    const int t = threadIdx.x + (q0 + q) * kRegBlock;
    const int l = t / N, k = t - l * N;
    S[regline<T, N>(l) + rpad<N>(k)] = z[q];
  }
  }
  __syncthreads();
  fft_reg_block<T, N, true>(S, tws);
  __syncthreads();
  pdl_trigger();
  const T inv_n = T(1) / T(N);
  constexpr int NH = N / 2;
  for (int t = threadIdx.x; t < nl * NH; t += kRegBlock) {
    const int l = t / NH, i0 = 2 * (t - l * NH);
    const int r0 = 2 * (line0 + l), r1 = r0 + 1;
    cplx<T> v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + h;
      const int src = mode == 1 ? ((i & 1) ? N - 1 - (i >> 1) : (i >> 1)) : i;
      v[h] = S[regline<T, N>(l) + rpad<N>(src)];
    }
    V wa, wb;
    wa.x = v[0].x * inv_n;
    wa.y = v[1].x * inv_n;
    wb.x = v[0].y * inv_n;
    wb.y = v[1].y * inv_n;
    *reinterpret_cast<V*>(data + (size_t)r0 * N + i0) = wa;
    if (r1 < rows) *reinterpret_cast<V*>(data + (size_t)r1 * N + i0) = wb;
  }
}

// z forward (see zfwd_kernel): complex lines of slot pairs along z at one y row.
template <typename T, int N>
__global__ void __launch_bounds__(kRegBlock, kRegMinBlocks<N>) zfwd_reg_kernel(T* __restrict__ data, int nx, int ny,
                                                           const cplx<T>* __restrict__ tw, int tile0) {
  pdl_wait();
  constexpr int P = regpitch<T, N>();
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* S = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tws = S + kRegLines * P;
  const int j = blockIdx.y;
  const int pair0 = (blockIdx.x + tile0) * kRegLines;
  const int np = min(kRegLines, nx / 2 - pair0);
  const size_t plane = (size_t)nx * ny;
  T* base = data + (size_t)nx * j + 2 * pair0;
  load_twiddles<T, N>(tws, tw);
  load_pair_tile<T, N>(S, base, plane, 2 * np);
  __syncthreads();
  fft_reg_block<T, N, false>(S, tws);
  __syncthreads();
  pdl_trigger();
  store_pair_tile<T, N>(base, plane, 2 * np, [&](int line, int p) -> cplx<T> {
    const cplx<T>* Z = S + regline<T, N>(line);
    if (pair0 + line > 0) return Z[rpad<N>(p)];
    // pair 0 holds two real sequences: split into two real-packed z spectra
    const int l = p == 0 ? 0 : (p == 1 ? N / 2 : p >> 1);
    const bool im = p >= 2 && (p & 1);
    const cplx<T> z = Z[rpad<N>(l)], zr = Z[rpad<N>(l == 0 ? 0 : N - l)];
    return im ? cplx<T>{T(0.5) * (z.y - zr.y), T(0.5) * (zr.x - z.x)}
              : cplx<T>{T(0.5) * (z.x + zr.x), T(0.5) * (z.y + zr.y)};
  });
}

// z inverse (see zinv_kernel).  Pair 0 arrives as two real-packed spectra in
// slots 0 and 1; the first block stages that line in a scratch line and
// rebuilds Z = Y0 + i Y1 into line 0.
template <typename T, int N>
__global__ void __launch_bounds__(kRegBlock, kRegMinBlocks<N>) zinv_reg_kernel(T* __restrict__ data, int nx, int ny,
                                                           const cplx<T>* __restrict__ tw, int tile0) {
  pdl_wait();
  constexpr int P = regpitch<T, N>();
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* S = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tws = S + kRegLines * P;
  cplx<T>* X = tws + N;   // scratch line (pair 0)
  const int j = blockIdx.y;
  const int pair0 = (blockIdx.x + tile0) * kRegLines;
  const int np = min(kRegLines, nx / 2 - pair0);
  const size_t plane = (size_t)nx * ny;
  T* base = data + (size_t)nx * j + 2 * pair0;
  load_twiddles<T, N>(tws, tw);
  load_pair_tile<T, N>(S, base, plane, 2 * np);
  __syncthreads();
  if (pair0 == 0) {
    for (int e = threadIdx.x; e < N; e += blockDim.x) X[rpad<N>(e)] = S[rpad<N>(e)];
    __syncthreads();
    for (int l = threadIdx.x; l < N; l += blockDim.x) {
      cplx<T> y0, y1;
      if (l == 0) {
        const cplx<T> a = X[rpad<N>(0)];
        y0 = {a.x, T(0)};
        y1 = {a.y, T(0)};
      } else if (2 * l == N) {
        const cplx<T> a = X[rpad<N>(1)];
        y0 = {a.x, T(0)};
        y1 = {a.y, T(0)};
      } else if (2 * l < N) {
        const cplx<T> a = X[rpad<N>(2 * l)], b = X[rpad<N>(2 * l + 1)];
        y0 = {a.x, b.x};
        y1 = {a.y, b.y};
      } else {
        const int q = N - l;
        const cplx<T> a = X[rpad<N>(2 * q)], b = X[rpad<N>(2 * q + 1)];
        y0 = {a.x, -b.x};
        y1 = {a.y, -b.y};
      }
      S[rpad<N>(l)] = {y0.x - y1.y, y0.y + y1.x};
    }
    __syncthreads();
  }
  fft_reg_block<T, N, true>(S, tws);
  __syncthreads();
  pdl_trigger();
  const T inv_n = T(1) / T(N);
  store_pair_tile<T, N>(base, plane, 2 * np, [&](int line, int k) -> cplx<T> {
    const cplx<T> v = S[regline<T, N>(line) + rpad<N>(k)];
    return {v.x * inv_n, v.y * inv_n};
  });
}

// Periodic y (see yspec_kernel): y DFT of slot pairs, eigenvalue division, inverse DFT.
template <typename T, int N>
__global__ void __launch_bounds__(kRegBlock, kRegMinBlocks<N>) yspec_reg_kernel(T* __restrict__ data, const YSpecArgs A,
                                                            const cplx<T>* __restrict__ tw,
                                                            const T* __restrict__ lamy,
                                                            const T* __restrict__ lamxz) {
  pdl_wait();
  constexpr int P = regpitch<T, N>();
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* S = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tws = S + kRegLines * P;
  const int s0 = blockIdx.x * 32;
  const int t = blockIdx.y;
  const int ns = min(32, A.nx - s0);
  const int nl = (ns + 1) / 2;
  T* base = data + s0 + (size_t)A.nx * A.ny * t;
  const size_t rs = (size_t)A.nx;
  load_twiddles<T, N>(tws, tw);
  load_pair_tile<T, N>(S, base, rs, ns);
  __syncthreads();
  fft_reg_block<T, N, false>(S, tws);
  __syncthreads();
  // x + z eigenvalues of the block's slot pairs and the y eigenvalues, staged once
  __shared__ T Lab[2 * kRegLines], Ly[N / 2 + 1];
  if (threadIdx.x < 2 * nl) {
    const int sa = s0 + threadIdx.x;
    const int sl = sa < A.nx ? sa : sa - 1;   // the odd tail's missing partner takes its neighbour's value
    Lab[threadIdx.x] = lamxz[lam_index_spec<T>(A, sl, t)];
  }
  for (int k = threadIdx.x; k <= N / 2; k += blockDim.x) Ly[k] = lamy[k];
  __syncthreads();
  constexpr int NH = N / 2 + 1;
  for (int e = threadIdx.x; e < nl * NH; e += blockDim.x) {
    const int l = e / NH, k = e - l * NH;
    const int kk = k == 0 ? 0 : N - k;
    const T La = Lab[2 * l], Lb = Lab[2 * l + 1];
    const T ly = Ly[k];
    const T ma = ly + La, mb = ly + Lb;
    const T ia = ma != T(0) ? T(1) / ma : T(0);
    const T ib = mb != T(0) ? T(1) / mb : T(0);
    const T cp = T(0.5) * (ia + ib), cm = T(0.5) * (ia - ib);
    cplx<T>* line = S + regline<T, N>(l);
    const cplx<T> z1 = line[rpad<N>(k)], z2 = line[rpad<N>(kk)];
    line[rpad<N>(k)] = {cp * z1.x + cm * z2.x, cp * z1.y - cm * z2.y};
    if (kk != k) line[rpad<N>(kk)] = {cp * z2.x + cm * z1.x, cp * z2.y - cm * z1.y};
  }
  __syncthreads();
  fft_reg_block<T, N, true>(S, tws);
  __syncthreads();
  pdl_trigger();
  const T inv_n = T(1) / T(N);
  store_pair_tile<T, N>(base, rs, ns, [&](int line, int jj) -> cplx<T> {
    const cplx<T> v = S[regline<T, N>(line) + rpad<N>(jj)];
    return {v.x * inv_n, v.y * inv_n};
  });
}

// ---------------------------------------------------------------------------
// Periodic y of 4096-row columns in three launches (the four-step decomposition
// 4096 = 64 x 64 across launches: n = 64 n1 + n2, k = k1 + 64 k2):
//   y4_outer<fwd>: for each n2, the 64-point DFT over n1 of rows 64 n1 + n2,
//                  times W_4096^{n2 k1}, back to row 64 k1 + n2;
//   y4_mid:        for each k1, the 64-point DFT over n2 of rows 64 k1 + n2
//                  gives X(k1 + 64 k2) in sub-line position k2; the eigenvalue
//                  division (see yspec_kernel) pairs X(k) with X(4096 - k),
//                  whose k1 is 64 - k1 (0 and 32 pair with themselves), so a
//                  block holds the sub-lines of k1 and 64 - k1 (block 0: 0 and
//                  32); the inverse 64-point DFT over k2 returns row 64 k1 + n2;
//   y4_outer<inv>: for each n2, times W_4096^{-n2 k1}, the inverse 64-point DFT
//                  over k1 and the factor 1/4096, back to row 64 n1 + n2.
// Every block moves 32 consecutive slots (16 slot pairs, 128 B of FP32 per row)
// of 128 rows: whole row segments instead of the few-slot columns that one
// block per 4096-row line would read.  Each launch holds 32 sub-lines of 64
// points (two row groups x 16 slot pairs), 8 transform threads per sub-line.
constexpr int kY4 = 64;   // 4096 = kY4 * kY4
constexpr int kY4Sub = 32;
// Sub-line s of the tile starts at 96 s + 8 (s mod 2) + s / 2 (complex entries; the padded
// 64-point line spans 71).  The 16 sub-lines a warp transposes start in 16 different 8-byte bank
// pairs, and the four lines a warp transforms pair up 8 bank pairs apart, so with FP32 entries
// neither the transposition nor the two in-line passes replay (a plain pitch of 73 put the lines'
// starts on the in-line stride of 9 and replayed the passes up to four times).
constexpr int kY4Pitch = 96;
__device__ __forceinline__ int y4line(int s) { return kY4Pitch * s + 8 * (s & 1) + (s >> 1); }

template <typename T>
size_t y4_smem_bytes() {
  return (size_t)(kY4Sub * kY4Pitch + kY4) * sizeof(cplx<T>);
}

// Slot-pair tile of the block: sub-line 16 g + m (g < 2) entry e (< 64) <-> global row row(g, e),
// slots 2m, 2m + 1; thread = (pair m, entries r0 + 16 q).
template <typename T, typename RowF, typename Mul>
__device__ __forceinline__ void y4_load(cplx<T>* S, const T* __restrict__ base, size_t rs, int nslots, RowF row,
                                        Mul mul) {
  const int m = threadIdx.x & 15, r0 = threadIdx.x >> 4;
  if (2 * m >= nslots) return;
  const bool whole = 2 * m + 1 < nslots;
  using V = typename Pair2<T>::V;
  cplx<T> v[2][4];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T* a = base + rs * row(g, r0 + 16 * q) + 2 * m;
      if (whole) {
        const V w = *reinterpret_cast<const V*>(a);
        v[g][q] = {w.x, w.y};
      } else {
        v[g][q] = {a[0], T(0)};
      }
    }
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int q = 0; q < 4; ++q) S[y4line(16 * g + m) + rpad<kY4>(r0 + 16 * q)] = mul(g, r0 + 16 * q, v[g][q]);
}

template <typename T, typename RowF, typename Val>
__device__ __forceinline__ void y4_store(T* __restrict__ base, size_t rs, int nslots, RowF row, Val value) {
  const int m = threadIdx.x & 15, r0 = threadIdx.x >> 4;
  if (2 * m >= nslots) return;
  const bool whole = 2 * m + 1 < nslots;
  using V = typename Pair2<T>::V;
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const cplx<T> o = value(g, m, r0 + 16 * q);
      T* a = base + rs * row(g, r0 + 16 * q) + 2 * m;
      if (whole) {
        V w;
        w.x = o.x;
        w.y = o.y;
        *reinterpret_cast<V*>(a) = w;
      } else {
        a[0] = o.x;
      }
    }
}

// tw: the 4096-entry table exp(-2 pi i e / 4096); blocks (slot tile, n2 pair, z position)
template <typename T, bool INV>
__global__ void __launch_bounds__(kRegBlock, sizeof(T) == 4 ? 5 : 4) y4_outer_kernel(T* __restrict__ data, int nx,
                                                                const cplx<T>* __restrict__ tw) {
  pdl_wait();
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* S = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tws = S + kY4Sub * kY4Pitch;
  const int s0 = blockIdx.x * 32;
  const int n2a = 2 * blockIdx.y;
  const int ns = min(32, nx - s0);
  T* base = data + s0 + (size_t)nx * (kY4 * kY4) * blockIdx.z;
  const size_t rs = (size_t)nx;
  if (threadIdx.x < kY4) tws[threadIdx.x] = tw[kY4 * threadIdx.x];
  auto row = [&](int g, int e) { return kY4 * e + n2a + g; };
  y4_load<T>(S, base, rs, ns, row, [&](int g, int e, cplx<T> v) {
    if (!INV) return v;
    cplx<T> w = tw[(n2a + g) * e];
    w.y = -w.y;
    return cmul(v, w);
  });
  __syncthreads();
  fft_reg_line<T, kY4, INV>(S + y4line(threadIdx.x >> 3), threadIdx.x & 7, tws);
  __syncthreads();
  pdl_trigger();
  const T inv_n = T(1) / T(kY4 * kY4);
  y4_store<T>(base, rs, ns, row, [&](int g, int m, int e) -> cplx<T> {
    const cplx<T> v = S[y4line(16 * g + m) + rpad<kY4>(e)];
    if (INV) return {v.x * inv_n, v.y * inv_n};
    return cmul(v, tw[(n2a + g) * e]);
  });
}

// blocks (slot tile, k1 pair b < 32, z position)
template <typename T>
__global__ void __launch_bounds__(kRegBlock, sizeof(T) == 4 ? 5 : 4) y4_mid_kernel(T* __restrict__ data, const YSpecArgs A,
                                                              const cplx<T>* __restrict__ tw,
                                                              const T* __restrict__ lamy,
                                                              const T* __restrict__ lamxz) {
  pdl_wait();
  constexpr int N = kY4 * kY4;
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* S = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tws = S + kY4Sub * kY4Pitch;
  __shared__ T Lab[32];
  const int s0 = blockIdx.x * 32;
  const int b = blockIdx.y;
  const int t = blockIdx.z;
  const int k1g0 = b, k1g1 = b == 0 ? kY4 / 2 : kY4 - b;
  const int ns = min(32, A.nx - s0);
  const int nl = (ns + 1) / 2;
  T* base = data + s0 + (size_t)A.nx * N * t;
  const size_t rs = (size_t)A.nx;
  if (threadIdx.x < kY4) tws[threadIdx.x] = tw[kY4 * threadIdx.x];
  if (threadIdx.x < 2 * nl) {
    const int sa = s0 + threadIdx.x;
    const int sl = sa < A.nx ? sa : sa - 1;   // the odd tail's missing partner takes its neighbour's value
    Lab[threadIdx.x] = lamxz[lam_index_spec<T>(A, sl, t)];
  }
  static_assert(kRegBlock == 256, "the eigenvalue step maps 256 threads to (k2 < 32, group, sub-line)");
  const T ly_own = lamy[((threadIdx.x >> 5) & 1 ? k1g1 : k1g0) + kY4 * (threadIdx.x & 31)];
  const T ly_mid = lamy[N / 2];
  auto row = [&](int g, int e) { return kY4 * (g ? k1g1 : k1g0) + e; };
  y4_load<T>(S, base, rs, ns, row, [](int, int, cplx<T> v) { return v; });
  __syncthreads();
  fft_reg_line<T, kY4, false>(S + y4line(threadIdx.x >> 3), threadIdx.x & 7, tws);
  __syncthreads();
  // sub-line 16 g + l position k2 holds X(k1_g + 64 k2); each pair (k, 4096 - k) is updated once,
  // by its lower k: every k2 < 32 of both groups, and k2 = 32 of group 0 when b = 0 (k = 2048).
  // Thread (k2, g) = (t mod 32, t / 32 mod 2) takes sub-lines l = t / 64 + 4 i; with its k fixed,
  // lamy[k] is read once.
  auto pair_update = [&](int l, int g, int gg, int k2, int q2, bool both, T ly) {
    const T La = Lab[2 * l], Lb = Lab[2 * l + 1];
    const T ma = ly + La, mb = ly + Lb;
    const T ia = ma != T(0) ? T(1) / ma : T(0);
    const T ib = mb != T(0) ? T(1) / mb : T(0);
    const T cp = T(0.5) * (ia + ib), cm = T(0.5) * (ia - ib);
    cplx<T>* p1 = S + y4line(16 * g + l) + rpad<kY4>(k2);
    cplx<T>* p2 = S + y4line(16 * gg + l) + rpad<kY4>(q2);
    const cplx<T> z1 = *p1, z2 = *p2;
    *p1 = {cp * z1.x + cm * z2.x, cp * z1.y - cm * z2.y};
    if (both) *p2 = {cp * z2.x + cm * z1.x, cp * z2.y - cm * z1.y};
  };
  {
    const int k2 = threadIdx.x & 31, g = (threadIdx.x >> 5) & 1;
    const int k1 = g ? k1g1 : k1g0;
    const int k = k1 + kY4 * k2;
    const int kk = (N - k) & (N - 1);
    const int gg = (kk & (kY4 - 1)) == k1 ? g : 1 - g;
    for (int l = threadIdx.x >> 6; l < nl; l += kRegBlock / 64) pair_update(l, g, gg, k2, kk / kY4, kk != k, ly_own);
    if (b == 0 && threadIdx.x < nl) pair_update(threadIdx.x, 0, 0, kY4 / 2, kY4 / 2, false, ly_mid);
  }
  __syncthreads();
  fft_reg_line<T, kY4, true>(S + y4line(threadIdx.x >> 3), threadIdx.x & 7, tws);
  __syncthreads();
  pdl_trigger();
  y4_store<T>(base, rs, ns, row, [&](int g, int m, int e) { return S[y4line(16 * g + m) + rpad<kY4>(e)]; });
}

// ---------------------------------------------------------------------------
// x transforms of 4096-point rows: one complex line (two rows) per block of 256
// threads, held in shared memory with one pad entry every 16 (entry i at
// i + i / 16) and transformed in place by three radix-16 Stockham passes
// (sub-transform sizes 1, 16, 256).  Thread j takes entries j + 256 r, r < 16,
// twiddles them by W^{r (j mod Ns)} of the 16 Ns-point stage, forms their
// 16-point DFT and, after the whole block has read its entries, writes them to
// (j / Ns) 16 Ns + (j mod Ns) + r Ns.  With the pad every read and every write
// of a half-warp touches 16 different bank pairs.
constexpr int kX4 = 4096;
__host__ __device__ constexpr int x4pad(int i) { return i + (i >> 4); }
template <typename T>
constexpr size_t x4_smem_bytes() {
  return (size_t)x4pad(kX4) * sizeof(cplx<T>);
}

template <typename T, bool INV>
__device__ __forceinline__ void fft4096_line(cplx<T>* L, const cplx<T>* __restrict__ tw) {
  const int j = threadIdx.x;
#pragma unroll
  for (int pass = 0; pass < 3; ++pass) {
    const int lg = 4 * pass;   // log2 of the sub-transform size Ns
    const int k = j & ((1 << lg) - 1);
    cplx<T> v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = L[x4pad(j + 256 * r)];
    if (pass > 0) {
#pragma unroll
      for (int r = 1; r < 16; ++r) {
        cplx<T> w = tw[(k * r) << (8 - lg)];   // exp(-2 pi i r k / (16 Ns))
        if (INV) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    dft16<T, INV>(v);
    __syncthreads();   // every entry of the pass read
    const int d = ((j >> lg) << (lg + 4)) + k;
#pragma unroll
    for (int r = 0; r < 16; ++r) L[x4pad(d + (r << lg))] = v[r];
    __syncthreads();
  }
}

// x forward of 4096-point rows (see xfwd_kernel: mode 0 real-packed DFT, 1 DCT-II; DIV forms the
// rows as the divergence of the predicted velocity)
template <typename T, bool DIV>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) xfwd4k_kernel(T* __restrict__ data, int rows, int mode,
                                                        const cplx<T>* __restrict__ tw,
                                                        const cplx<T>* __restrict__ dtw, const DivArgs<T> dv) {
  pdl_wait();
  constexpr int N = kX4;
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* L = reinterpret_cast<cplx<T>*>(smem_raw);
  const int r0 = 2 * blockIdx.x, r1 = r0 + 1;
  const bool two = r1 < rows;
  int ja = 0, ka = 0, jb = 0, kb = 0;
  if constexpr (DIV) {
    ka = r0 / dv.g.ny;
    ja = r0 - ka * dv.g.ny;
    kb = r1 / dv.g.ny;
    jb = r1 - kb * dv.g.ny;
  }
  bool done = false;
  if constexpr (DIV) {
    if (dv.vec4 && mode == 0 && dv.g.dim == 2 && sizeof(T) == 4) {
      // 2-D FP32 rows: the raw loads of two quads of both rows (u with its right neighbour, v at
      // j and j + 1) issued together before any arithmetic (the divergence as div4_at forms it)
      const Geom<T>& g = dv.g;
      const int ey = g.ext(1, 1);
      const int jb2 = two ? jb : ja;
      const int jr[2] = {ja, jb2};
      const T ih[2] = {g.ihy[ja], g.ihy[jb2]};
#pragma unroll
      for (int u0 = 0; u0 < 4; u0 += 2) {
        Vec4<T> xu[2][2], xv0[2][2], xv1[2][2];
        T xe[2][2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const int i0 = 4 * (threadIdx.x + 256 * (u0 + b));
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = jr[h];
            const T* ur = dv.u[0] + (size_t)N * j;
            xu[b][h] = ld4(ur + i0);
            xe[b][h] = __ldg(ur + (i0 + 4 < N ? i0 + 4 : 0));
            const int jp = j + 1 < ey ? j + 1 : 0;
            xv0[b][h] = ld4(dv.u[1] + (size_t)N * j + i0);
            xv1[b][h] = ld4(dv.u[1] + (size_t)N * jp + i0);
          }
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const int i0 = 4 * (threadIdx.x + 256 * (u0 + b));
          T d[2][4];
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              T sv = ((c < 3 ? xu[b][h].v[c + 1] : xe[b][h]) - xu[b][h].v[c]) * g.ihx;
              sv += (xv1[b][h].v[c] - xv0[b][h].v[c]) * ih[h];
              d[h][c] = (h == 0 || two) ? sv : T(0);
            }
#pragma unroll
          for (int c = 0; c < 4; ++c) L[x4pad(i0 + c)] = {d[0][c], d[1][c]};
        }
      }
      done = true;
    } else if (dv.vec4 && mode == 0) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i0 = 4 * (threadIdx.x + 256 * u);
        const Vec4<T> da = div4_at(dv, i0, ja, ka);
        Vec4<T> db = {{T(0), T(0), T(0), T(0)}};
        if (two) db = div4_at(dv, i0, jb, kb);
#pragma unroll
        for (int e = 0; e < 4; ++e) L[x4pad(i0 + e)] = {da.v[e], db.v[e]};
      }
      done = true;
    }
  }
  if (!done) {
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
      const int i = threadIdx.x + 256 * q;
      T va, vb = T(0);
      if constexpr (DIV) {
        va = div_at(dv, i, ja, ka);
        if (two) vb = div_at(dv, i, jb, kb);
      } else {
        va = data[(size_t)r0 * N + i];
        if (two) vb = data[(size_t)r1 * N + i];
      }
      const int dst = mode == 1 ? ((i & 1) ? N - 1 - (i >> 1) : (i >> 1)) : i;   // DCT: even forward, odd reversed
      L[x4pad(dst)] = {va, vb};
    }
  }
  __syncthreads();
  fft4096_line<T, false>(L, tw);
  pdl_trigger();
  using V = typename Pair2<T>::V;
  for (int t = threadIdx.x; t < N / 2; t += 256) {
    const int s0 = 2 * t;
    T oa[2], ob[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int s = s0 + h;
      int m;
      bool im = false;
      if (mode == 0) {
        m = s == 0 ? 0 : (s == 1 ? N / 2 : s >> 1);
        im = s >= 2 && (s & 1);
      } else {
        m = s;
      }
      const cplx<T> z = L[x4pad(m)], zr = L[x4pad(m == 0 ? 0 : N - m)];
      const cplx<T> xa = {T(0.5) * (z.x + zr.x), T(0.5) * (z.y - zr.y)};
      const cplx<T> xb = {T(0.5) * (z.y + zr.y), T(0.5) * (zr.x - z.x)};
      if (mode == 0) {
        oa[h] = im ? xa.y : xa.x;
        ob[h] = im ? xb.y : xb.x;
      } else {
        const cplx<T> w = dtw[m];
        oa[h] = w.x * xa.x - w.y * xa.y;
        ob[h] = w.x * xb.x - w.y * xb.y;
      }
    }
    V wa, wb;
    wa.x = oa[0];
    wa.y = oa[1];
    wb.x = ob[0];
    wb.y = ob[1];
    *reinterpret_cast<V*>(data + (size_t)r0 * N + s0) = wa;
    if (two) *reinterpret_cast<V*>(data + (size_t)r1 * N + s0) = wb;
  }
}

// x inverse of 4096-point rows (see xinv_kernel)
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) xinv4k_kernel(T* __restrict__ data, int rows, int mode,
                                                        const cplx<T>* __restrict__ tw,
                                                        const cplx<T>* __restrict__ dtw) {
  pdl_wait();
  constexpr int N = kX4;
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* L = reinterpret_cast<cplx<T>*>(smem_raw);
  const int r0 = 2 * blockIdx.x, r1 = r0 + 1;
  const bool two = r1 < rows;
  const T* ra = data + (size_t)r0 * N;
  const T* rb = data + (size_t)r1 * N;
  using V = typename Pair2<T>::V;
  if (mode == 0) {
    // Hermitian spectra from real-packed rows: the slot pair (2k, 2k + 1), 0 < k < N/2, read once
    // as one vector gives entries k and N - k (complex conjugates of each other); slot pair 0
    // holds the real X[0] and X[N/2].  Four pairs of both rows are loaded before any is stored.
#pragma unroll
    for (int q0 = 0; q0 < 8; q0 += 4) {
      V pa[4], pb[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int k = threadIdx.x + 256 * (q0 + c);
        pa[c] = *reinterpret_cast<const V*>(ra + 2 * k);
        pb[c].x = pb[c].y = T(0);
        if (two) pb[c] = *reinterpret_cast<const V*>(rb + 2 * k);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int k = threadIdx.x + 256 * (q0 + c);
        if (k == 0) {
          L[x4pad(0)] = {pa[c].x, pb[c].x};          // XA + i XB, both real
          L[x4pad(N / 2)] = {pa[c].y, pb[c].y};
        } else {
          L[x4pad(k)] = {pa[c].x - pb[c].y, pa[c].y + pb[c].x};
          L[x4pad(N - k)] = {pa[c].x + pb[c].y, pb[c].x - pa[c].y};
        }
      }
    }
  } else {
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
      const int k = threadIdx.x + 256 * q;
      // V[k] = exp(i pi k / 2N) (X[k] - i X[N-k]), X[N] = 0
      const cplx<T> w = cconj(dtw[k]);
      const T a1 = ra[k], a2 = k ? ra[N - k] : T(0);
      const cplx<T> xa = cmul(w, cplx<T>{a1, -a2});
      cplx<T> xb = {T(0), T(0)};
      if (two) {
        const T b1 = rb[k], b2 = k ? rb[N - k] : T(0);
        xb = cmul(w, cplx<T>{b1, -b2});
      }
      L[x4pad(k)] = {xa.x - xb.y, xa.y + xb.x};   // XA + i XB
    }
  }
  __syncthreads();
  fft4096_line<T, true>(L, tw);
  pdl_trigger();
  const T inv_n = T(1) / T(N);
  for (int t = threadIdx.x; t < N / 2; t += 256) {
    const int i0 = 2 * t;
    cplx<T> v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + h;
      const int src = mode == 1 ? ((i & 1) ? N - 1 - (i >> 1) : (i >> 1)) : i;
      v[h] = L[x4pad(src)];
    }
    V wa, wb;
    wa.x = v[0].x * inv_n;
    wa.y = v[1].x * inv_n;
    wb.x = v[0].y * inv_n;
    wb.y = v[1].y * inv_n;
    *reinterpret_cast<V*>(data + (size_t)r0 * N + i0) = wa;
    if (two) *reinterpret_cast<V*>(data + (size_t)r1 * N + i0) = wb;
  }
}

// ---------------------------------------------------------------------------
// x and z transforms of one y position j per block (3-D, FP32 fields, nx = nz = N
// of 64 or 128, periodic x and z).  The x-z plane of a y position (N rows k of N
// values, 16 or 64 KB) fits in shared memory, so both directions are done in one
// pass over the field instead of the two of the x and z kernels:
//   forward: rows (divergence formed on the fly, or read) -> N/2 row-pair lines
//            (rows 2l, 2l + 1 as real and imaginary parts), x DFT, real-packed
//            split written as N/2 slot-pair lines along z, z DFT, written out in
//            the layout of zfwd_reg_kernel (pair 0 split into two real-packed z
//            spectra);
//   inverse: the mirror image (zinv_reg_kernel, then xinv_reg_kernel with the
//            rows paired along z instead of along y), one 1 / N^2 at the end.
// Each line is transformed by 8 threads (fft_reg_line); 8 N threads per block,
// half of them transform while the other half idles, all of them move data.
// Line s of each half of the plane starts at xzpitch s + 8 (s mod 2) + (s / 2 mod 16): lines
// 32 apart repeat the skew, every 32 consecutive lines start twice in each of the 16 8-byte bank
// pairs (the slot-pair transpositions stay conflict-free) and the four lines a warp transforms
// start 8 bank pairs apart, so the in-line FFT passes do not replay either (with the plain pitch
// N + N / R1 + 1 = 9 mod 16 they replayed up to three times)
template <int N>
__host__ __device__ constexpr int xzpitch() {
  return (N + N / RegPlan<N>::R1 + 23 + 15) / 16 * 16;   // padded line + largest skew, 16-aligned
}
template <int N>
__device__ __forceinline__ int xzline(int s) {
  return xzpitch<N>() * s + 8 * (s & 1) + ((s >> 1) & 15);
}
template <int N>
constexpr size_t plane_smem_bytes() {
  return (size_t)(N * xzpitch<N>() + N) * sizeof(cplx<float>);
}

template <int N, bool DIV>
__global__ void __launch_bounds__(8 * N, 1) xzfwd_plane_kernel(float* __restrict__ data, int ny,
                                                               const cplx<float>* __restrict__ tw,
                                                               const DivArgs<float> dv) {
  pdl_wait();
  using T = float;
  constexpr int NL = N / 2, NT = 8 * N, TPL = RegPlan<N>::TPL;
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* A = reinterpret_cast<cplx<T>*>(smem_raw);   // z lines: slot pair c, entry k
  cplx<T>* B = A + NL * xzpitch<N>();   // x lines: row pair l, entry i
  cplx<T>* tws = B + NL * xzpitch<N>();
  const int j = blockIdx.x;
  const size_t rs = (size_t)N * ny;   // between z positions
  T* base = data + (size_t)N * j;
  for (int e = threadIdx.x; e < N; e += NT) tws[e] = tw[e];
  // row pairs (2l, 2l + 1) of the plane as quads of x positions, stored as complex pairs
  constexpr int NQ = N * N / 8 / NT;   // row-pair quads per thread
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int e = threadIdx.x + NT * q;
    const int l = e / (N / 4), i0 = 4 * (e - l * (N / 4));
    float va[4], vb[4];
    if constexpr (DIV) {
      // D u* at rows k0 = 2l and k1 = 2l + 1 (as div4_at): the rows share the w quad of k1, and the
      // x neighbour of a quad's last cell is the next lane's first (a row's quads fill N / 4
      // consecutive lanes, periodic in x)
      const Geom<T>& g = dv.g;
      const int k0 = 2 * l, k1 = k0 + 1, k2 = k1 + 1 < g.nz ? k1 + 1 : 0;
      const Vec4<T> ua = ld4(dv.u[0] + rs * k0 + (size_t)N * j + i0);
      const Vec4<T> ub = ld4(dv.u[0] + rs * k1 + (size_t)N * j + i0);
      const int ey = g.ext(1, 1);
      const int jp = j + 1 < ey ? j + 1 : 0;
      const T* vp = dv.u[1] + i0;
      const size_t vs = (size_t)N * ey;
      const Vec4<T> v0a = ld4(vp + vs * k0 + (size_t)N * j), v1a = ld4(vp + vs * k0 + (size_t)N * jp);
      const Vec4<T> v0b = ld4(vp + vs * k1 + (size_t)N * j), v1b = ld4(vp + vs * k1 + (size_t)N * jp);
      const T* wp = dv.u[2] + (size_t)N * j + i0;
      const Vec4<T> w0 = ld4(wp + rs * k0), w1 = ld4(wp + rs * k1), w2 = ld4(wp + rs * k2);
      constexpr int Q = N / 4;
      const int lane = threadIdx.x & 31;
      const int nb = (lane & ~(Q - 1)) | ((lane + 1) & (Q - 1));
      const T ea = __shfl_sync(0xffffffffu, ua.v[0], nb), eb = __shfl_sync(0xffffffffu, ub.v[0], nb);
      const T ih = g.ihy[j];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        va[c] = ((c < 3 ? ua.v[c + 1] : ea) - ua.v[c]) * g.ihx;
        vb[c] = ((c < 3 ? ub.v[c + 1] : eb) - ub.v[c]) * g.ihx;
        va[c] += (v1a.v[c] - v0a.v[c]) * ih;
        vb[c] += (v1b.v[c] - v0b.v[c]) * ih;
        va[c] += (w1.v[c] - w0.v[c]) * g.ihz;
        vb[c] += (w2.v[c] - w1.v[c]) * g.ihz;
      }
    } else {
      const float4 da = *reinterpret_cast<const float4*>(base + rs * (2 * l) + i0);
      const float4 db = *reinterpret_cast<const float4*>(base + rs * (2 * l + 1) + i0);
      va[0] = da.x; va[1] = da.y; va[2] = da.z; va[3] = da.w;
      vb[0] = db.x; vb[1] = db.y; vb[2] = db.z; vb[3] = db.w;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) B[xzline<N>(l) + rpad<N>(i0 + c)] = {va[c], vb[c]};
  }
  __syncthreads();
  if (threadIdx.x < NL * TPL) fft_reg_line<T, N, false>(B + xzline<N>(threadIdx.x / TPL), threadIdx.x % TPL, tws);
  __syncthreads();
  // real-packed split of rows 2l, 2l + 1: slot pair c (slots 2c, 2c + 1) of row k -> A[c][k]
  for (int e = threadIdx.x; e < NL * NL; e += NT) {
    const int l = e / NL, c = e - l * NL;
    const cplx<T>* line = B + xzline<N>(l);
    cplx<T> oa, ob;
    if (c == 0) {   // slots 0 and 1: the real modes 0 and N / 2
      const cplx<T> z0 = line[rpad<N>(0)], zh = line[rpad<N>(N / 2)];
      oa = {z0.x, zh.x};
      ob = {z0.y, zh.y};
    } else {
      const cplx<T> z = line[rpad<N>(c)], zr = line[rpad<N>(N - c)];
      oa = {T(0.5) * (z.x + zr.x), T(0.5) * (z.y - zr.y)};   // XA = (Z + conj Zr) / 2
      ob = {T(0.5) * (z.y + zr.y), T(0.5) * (zr.x - z.x)};   // XB = (Z - conj Zr) / (2 i)
    }
    A[xzline<N>(c) + rpad<N>(2 * l)] = oa;
    A[xzline<N>(c) + rpad<N>(2 * l + 1)] = ob;
  }
  __syncthreads();
  if (threadIdx.x < NL * TPL) fft_reg_line<T, N, false>(A + xzline<N>(threadIdx.x / TPL), threadIdx.x % TPL, tws);
  __syncthreads();
  pdl_trigger();
  constexpr int NE = N * NL / NT;   // slot pairs per thread
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = threadIdx.x + NT * q;
    const int k = e / NL, c = e - k * NL;
    cplx<T> o;
    if (c > 0) {
      o = A[xzline<N>(c) + rpad<N>(k)];
    } else {   // pair 0 holds two real sequences: split into two real-packed z spectra
      const int m = k == 0 ? 0 : (k == 1 ? N / 2 : k >> 1);
      const bool im = k >= 2 && (k & 1);
      const cplx<T> z = A[rpad<N>(m)], zr = A[rpad<N>(m == 0 ? 0 : N - m)];
      o = im ? cplx<T>{T(0.5) * (z.y - zr.y), T(0.5) * (zr.x - z.x)}
             : cplx<T>{T(0.5) * (z.x + zr.x), T(0.5) * (z.y + zr.y)};
    }
    *reinterpret_cast<float2*>(base + rs * k + 2 * c) = make_float2(o.x, o.y);
  }
}

template <int N>
__global__ void __launch_bounds__(8 * N, 1) zxinv_plane_kernel(float* __restrict__ data, int ny,
                                                               const cplx<float>* __restrict__ tw) {
  pdl_wait();
  using T = float;
  constexpr int NL = N / 2, NT = 8 * N, TPL = RegPlan<N>::TPL;
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* A = reinterpret_cast<cplx<T>*>(smem_raw);   // z lines: slot pair c, entry k
  cplx<T>* B = A + NL * xzpitch<N>();   // x lines: row pair l, entry i
  cplx<T>* tws = B + NL * xzpitch<N>();
  const int j = blockIdx.x;
  const size_t rs = (size_t)N * ny;
  T* base = data + (size_t)N * j;
  for (int e = threadIdx.x; e < N; e += NT) tws[e] = tw[e];
  constexpr int NE = N * NL / NT;
  float2 v[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = threadIdx.x + NT * q;
    const int k = e / NL, c = e - k * NL;
    v[q] = *reinterpret_cast<const float2*>(base + rs * k + 2 * c);
  }
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = threadIdx.x + NT * q;
    const int k = e / NL, c = e - k * NL;
    A[xzline<N>(c) + rpad<N>(k)] = {v[q].x, v[q].y};
    if (c == 0) B[rpad<N>(k)] = {v[q].x, v[q].y};   // pair 0 kept aside for its rebuild
  }
  __syncthreads();
  // pair 0: the two real-packed z spectra Y0 (slot 0), Y1 (slot 1) -> Z = Y0 + i Y1
  for (int l = threadIdx.x; l < N; l += NT) {
    cplx<T> y0, y1;
    if (l == 0 || 2 * l == N) {
      const cplx<T> a = B[rpad<N>(l == 0 ? 0 : 1)];
      y0 = {a.x, T(0)};
      y1 = {a.y, T(0)};
    } else {
      const int q = 2 * l < N ? l : N - l;
      const T sg = 2 * l < N ? T(1) : T(-1);
      const cplx<T> a = B[rpad<N>(2 * q)], b = B[rpad<N>(2 * q + 1)];
      y0 = {a.x, sg * b.x};
      y1 = {a.y, sg * b.y};
    }
    A[rpad<N>(l)] = {y0.x - y1.y, y0.y + y1.x};
  }
  __syncthreads();
  if (threadIdx.x < NL * TPL) fft_reg_line<T, N, true>(A + xzline<N>(threadIdx.x / TPL), threadIdx.x % TPL, tws);
  __syncthreads();
  // x lines: row pair l (rows 2l, 2l + 1), entry kx = XA + i XB, the Hermitian spectra of the two
  // rows from their real-packed slots (slots 2c, 2c + 1 of row k are A[c][k])
  for (int e = threadIdx.x; e < NL * N; e += NT) {
    const int l = e / N, kx = e - l * N;
    const int kk = 2 * kx <= N ? kx : N - kx;
    const int c = 2 * kk == N ? 0 : kk;
    const cplx<T> pa = A[xzline<N>(c) + rpad<N>(2 * l)], pb = A[xzline<N>(c) + rpad<N>(2 * l + 1)];
    cplx<T> xa, xb;
    if (kx == 0) {
      xa = {pa.x, T(0)};
      xb = {pb.x, T(0)};
    } else if (2 * kx == N) {
      xa = {pa.y, T(0)};
      xb = {pb.y, T(0)};
    } else if (2 * kx < N) {
      xa = pa;
      xb = pb;
    } else {
      xa = {pa.x, -pa.y};
      xb = {pb.x, -pb.y};
    }
    B[xzline<N>(l) + rpad<N>(kx)] = {xa.x - xb.y, xa.y + xb.x};
  }
  __syncthreads();
  if (threadIdx.x < NL * TPL) fft_reg_line<T, N, true>(B + xzline<N>(threadIdx.x / TPL), threadIdx.x % TPL, tws);
  __syncthreads();
  pdl_trigger();
  const T sc = T(1) / T(N * N);
  constexpr int NQ = N * N / 8 / NT;   // row-pair quads per thread
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int e = threadIdx.x + NT * q;
    const int l = e / (N / 4), i0 = 4 * (e - l * (N / 4));
    cplx<T> z[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) z[c] = B[xzline<N>(l) + rpad<N>(i0 + c)];
    *reinterpret_cast<float4*>(base + rs * (2 * l) + i0) =
        make_float4(z[0].x * sc, z[1].x * sc, z[2].x * sc, z[3].x * sc);
    *reinterpret_cast<float4*>(base + rs * (2 * l + 1) + i0) =
        make_float4(z[0].y * sc, z[1].y * sc, z[2].y * sc, z[3].y * sc);
  }
}

// The same fused x and z transforms with each y position's plane split over a
// cluster of two blocks (rank r): block r holds the row pairs l and the slot
// pairs c of its half (N / 4 lines of each kind) and transforms them with all
// of its 2 N threads (8 per line).  Forward: the block's rows through the x
// DFT, the real-packed split stored into the slot-pair lines of whichever
// block owns the slot pair (the peer's through distributed shared memory),
// a cluster barrier, the z DFT of its own slot pairs.  Inverse: its slot pairs
// through the z DFT, a cluster barrier, each row pair gathered from both
// blocks' slot-pair lines, the x DFT of its own rows.  Twice the blocks of
// the one-block form (all SMs busy at 128^3) and no idle threads in the
// transform passes, yet slower at 128^3 (20.5 and 25 us per launch against
// 16.5 and 14.4, and less overlap between launches): the one-block form is
// the default.
template <int N>
constexpr size_t plane_pair_smem_bytes() {
  return (size_t)(N / 2 * rpitch<N>() + N) * sizeof(cplx<float>);
}

template <int N, bool DIV>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(2 * N)
    xzfwd_pair_kernel(float* __restrict__ data, int ny, const cplx<float>* __restrict__ tw, const DivArgs<float> dv) {
  cluster_arrive_relaxed();   // this block runs: its shared memory may take the peer's stores
  pdl_wait();
  using T = float;
  constexpr int P = rpitch<N>(), NL = N / 2, NH = N / 4, NT = 2 * N, TPL = RegPlan<N>::TPL;
  static_assert(NH * TPL == NT, "one transform thread group per line");
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* A = reinterpret_cast<cplx<T>*>(smem_raw);   // own slot pairs c = NH r + cl, entry k
  cplx<T>* B = A + NH * P;                              // own row pairs l = NH r + ll, entry i
  cplx<T>* tws = B + NH * P;
  const int r = (int)cluster_rank();
  const int j = blockIdx.x >> 1;
  const size_t rs = (size_t)N * ny;
  T* base = data + (size_t)N * j;
  for (int e = threadIdx.x; e < N; e += NT) tws[e] = tw[e];
  // own rows k = N r / 2 + kk as quads of x positions
  constexpr int NQ = N / 16;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int e = threadIdx.x + NT * q;
    const int kk = e / (N / 4), i0 = 4 * (e - kk * (N / 4));
    const int k = NL * r + kk;
    float v[4];
    if constexpr (DIV) {
      const Vec4<T> d = div4_at(dv, i0, j, k);
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] = d.v[c];
    } else {
      const float4 d = *reinterpret_cast<const float4*>(base + rs * k + i0);
      v[0] = d.x; v[1] = d.y; v[2] = d.z; v[3] = d.w;
    }
    T* dst = reinterpret_cast<T*>(B + (kk >> 1) * P);
#pragma unroll
    for (int c = 0; c < 4; ++c) dst[2 * rpad<N>(i0 + c) + (kk & 1)] = v[c];
  }
  __syncthreads();
  fft_reg_line<T, N, false>(B + (threadIdx.x / TPL) * P, threadIdx.x % TPL, tws);
  __syncthreads();
  cluster_wait();   // the peer runs: its slot-pair lines may be written
  const uint32_t A_own = smem_u32(A), A_peer = map_peer(A_own, (uint32_t)(r ^ 1));
  for (int e = threadIdx.x; e < NH * NL; e += NT) {
    const int ll = e / NL, c = e - ll * NL;
    const int l = NH * r + ll;
    const cplx<T>* line = B + ll * P;
    cplx<T> oa, ob;
    if (c == 0) {
      const cplx<T> z0 = line[rpad<N>(0)], zh = line[rpad<N>(N / 2)];
      oa = {z0.x, zh.x};
      ob = {z0.y, zh.y};
    } else {
      const cplx<T> z = line[rpad<N>(c)], zr = line[rpad<N>(N - c)];
      oa = {T(0.5) * (z.x + zr.x), T(0.5) * (z.y - zr.y)};
      ob = {T(0.5) * (z.y + zr.y), T(0.5) * (zr.x - z.x)};
    }
    const int owner = c / NH, cl = c - owner * NH;
    const uint32_t at = (owner == r ? A_own : A_peer) + (uint32_t)((cl * P + rpad<N>(2 * l)) * sizeof(cplx<T>));
    st_cluster_f2(at, oa.x, oa.y);
    st_cluster_f2(at + (uint32_t)((rpad<N>(2 * l + 1) - rpad<N>(2 * l)) * sizeof(cplx<T>)), ob.x, ob.y);
  }
  cluster_arrive();   // this block's stores into both blocks' lines are done
  cluster_wait();     // and the peer's
  fft_reg_line<T, N, false>(A + (threadIdx.x / TPL) * P, threadIdx.x % TPL, tws);
  __syncthreads();
  pdl_trigger();
  constexpr int NE = N / 8;   // slot pairs per thread
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = threadIdx.x + NT * q;
    const int k = e / NH, cl = e - k * NH;
    const int c = NH * r + cl;
    cplx<T> o;
    if (c > 0) {
      o = A[cl * P + rpad<N>(k)];
    } else {   // pair 0: two real-packed z spectra
      const int m = k == 0 ? 0 : (k == 1 ? N / 2 : k >> 1);
      const bool im = k >= 2 && (k & 1);
      const cplx<T> z = A[rpad<N>(m)], zr = A[rpad<N>(m == 0 ? 0 : N - m)];
      o = im ? cplx<T>{T(0.5) * (z.y - zr.y), T(0.5) * (zr.x - z.x)}
             : cplx<T>{T(0.5) * (z.x + zr.x), T(0.5) * (z.y + zr.y)};
    }
    *reinterpret_cast<float2*>(base + rs * k + 2 * c) = make_float2(o.x, o.y);
  }
}

template <int N>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(2 * N)
    zxinv_pair_kernel(float* __restrict__ data, int ny, const cplx<float>* __restrict__ tw) {
  pdl_wait();
  using T = float;
  constexpr int P = rpitch<N>(), NL = N / 2, NH = N / 4, NT = 2 * N, TPL = RegPlan<N>::TPL;
  static_assert(NH * TPL == NT, "one transform thread group per line");
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* A = reinterpret_cast<cplx<T>*>(smem_raw);   // own slot pairs c = NH r + cl, entry k
  cplx<T>* B = A + NH * P;                              // own row pairs l = NH r + ll, entry i
  cplx<T>* tws = B + NH * P;
  const int r = (int)cluster_rank();
  const int j = blockIdx.x >> 1;
  const size_t rs = (size_t)N * ny;
  T* base = data + (size_t)N * j;
  for (int e = threadIdx.x; e < N; e += NT) tws[e] = tw[e];
  constexpr int NE = N / 8;
  float2 v[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = threadIdx.x + NT * q;
    const int k = e / NH, cl = e - k * NH;
    v[q] = *reinterpret_cast<const float2*>(base + rs * k + 2 * (NH * r + cl));
  }
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = threadIdx.x + NT * q;
    const int k = e / NH, cl = e - k * NH;
    A[cl * P + rpad<N>(k)] = {v[q].x, v[q].y};
    if (r == 0 && cl == 0) B[rpad<N>(k)] = {v[q].x, v[q].y};   // pair 0 kept aside for its rebuild
  }
  __syncthreads();
  if (r == 0) {   // pair 0: Y0 (slot 0), Y1 (slot 1) real-packed -> Z = Y0 + i Y1
    for (int l = threadIdx.x; l < N; l += NT) {
      cplx<T> y0, y1;
      if (l == 0 || 2 * l == N) {
        const cplx<T> a = B[rpad<N>(l == 0 ? 0 : 1)];
        y0 = {a.x, T(0)};
        y1 = {a.y, T(0)};
      } else {
        const int q = 2 * l < N ? l : N - l;
        const T sg = 2 * l < N ? T(1) : T(-1);
        const cplx<T> a = B[rpad<N>(2 * q)], b = B[rpad<N>(2 * q + 1)];
        y0 = {a.x, sg * b.x};
        y1 = {a.y, sg * b.y};
      }
      A[rpad<N>(l)] = {y0.x - y1.y, y0.y + y1.x};
    }
  }
  __syncthreads();
  fft_reg_line<T, N, true>(A + (threadIdx.x / TPL) * P, threadIdx.x % TPL, tws);
  cluster_arrive();   // this block's slot-pair lines are final
  cluster_wait();     // and the peer's
  const uint32_t A_own = smem_u32(A), A_peer = map_peer(A_own, (uint32_t)(r ^ 1));
  constexpr int RE = NH * N / NT, RB = 4;   // entries per thread, in batches of RB loads in flight
  static_assert(RE % RB == 0, "whole batches");
#pragma unroll
  for (int q0 = 0; q0 < RE; q0 += RB) {
    float2 pa[RB], pb[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int e = threadIdx.x + NT * (q0 + u);
      const int ll = e / N, kx = e - ll * N;
      const int l = NH * r + ll;
      const int kk = 2 * kx <= N ? kx : N - kx;
      const int c = 2 * kk == N ? 0 : kk;
      const int owner = c / NH, cl = c - owner * NH;
      const uint32_t at = (owner == r ? A_own : A_peer) + (uint32_t)((cl * P + rpad<N>(2 * l)) * sizeof(cplx<T>));
      pa[u] = ld_cluster_f2(at);
      pb[u] = ld_cluster_f2(at + (uint32_t)((rpad<N>(2 * l + 1) - rpad<N>(2 * l)) * sizeof(cplx<T>)));
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int e = threadIdx.x + NT * (q0 + u);
      const int ll = e / N, kx = e - ll * N;
      cplx<T> xa, xb;
      if (kx == 0) {
        xa = {pa[u].x, T(0)};
        xb = {pb[u].x, T(0)};
      } else if (2 * kx == N) {
        xa = {pa[u].y, T(0)};
        xb = {pb[u].y, T(0)};
      } else if (2 * kx < N) {
        xa = {pa[u].x, pa[u].y};
        xb = {pb[u].x, pb[u].y};
      } else {
        xa = {pa[u].x, -pa[u].y};
        xb = {pb[u].x, -pb[u].y};
      }
      B[ll * P + rpad<N>(kx)] = {xa.x - xb.y, xa.y + xb.x};
    }
  }
  cluster_arrive();   // the peer's lines are no longer read by this block
  __syncthreads();
  fft_reg_line<T, N, true>(B + (threadIdx.x / TPL) * P, threadIdx.x % TPL, tws);
  __syncthreads();
  pdl_trigger();
  const T sc = T(1) / T(N * N);
  constexpr int NQ = N / 16;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int e = threadIdx.x + NT * q;
    const int kk = e / (N / 4), i0 = 4 * (e - kk * (N / 4));
    const int k = NL * r + kk;
    const T* src = reinterpret_cast<const T*>(B + (kk >> 1) * P);
    float4 o;
    o.x = src[2 * rpad<N>(i0) + (kk & 1)] * sc;
    o.y = src[2 * rpad<N>(i0 + 1) + (kk & 1)] * sc;
    o.z = src[2 * rpad<N>(i0 + 2) + (kk & 1)] * sc;
    o.w = src[2 * rpad<N>(i0 + 3) + (kk & 1)] * sc;
    *reinterpret_cast<float4*>(base + rs * k + i0) = o;
  }
  cluster_wait();   // the peer no longer reads this block's lines: its shared memory may go
}
