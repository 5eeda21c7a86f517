// fft.cuh -- 2D/3D real-to-complex FFT for sm_103a in two HBM passes.
//
// Transform convention (the spectral collocation of Sec. 3.2): forward
//   F_k = sum_j f_j exp(-2 pi i j.k / N), inverse with +i and 1/N.
//
// Decomposition ("four-step" split of the y axis, Ny = Y1 * Y2 with Y2 = min(Ny, 16),
// y = n1 + Y1 * n2, ky = k2 + Y2 * k1):
//   pass A (one CTA per z-block of ZB planes and residue n1): the Y2 rows y = n1 + Y1*j of
//     each plane are real-to-complex transformed along x (two real rows packed into one
//     complex row), then Y2-point DFTs across the rows give k2, then the twiddle
//     w_Ny^(n1 k2).  Out: intermediate I[k2][kx][n1][z].
//   pass B (one CTA per kx and k2): the Y1-point DFT over n1 gives k1, the Nz-point DFT over
//     z gives kz.  The spectrum sits in registers; a pointwise spectral operator runs there
//     (the ETD update), and the results go straight back through the inverse pass B.
// The spectral layout is therefore S[k2][kx][k1][kz] (complex), the same index map as the
// intermediate, so stored spectra are read and written by pass B in contiguous chunks.
//
// Long transforms (x in pass A, z in pass B) run on a team of S lanes of one warp holding
// R = L/S values each: an R-point DFT in registers, a twiddle w_L^(t k1), and log2 S
// radix-2 decimation-in-frequency stages across the lanes by warp shuffles, which leave
// lane t holding X[k1 + R * bitrev(t)].  The inverse runs the conjugate-transposed stages
// in reverse order, so it takes that bit-reversed layout and returns natural order (and
// coalesced stores).  Short transforms across rows (Y1, Y2 <= 16) run one column per
// thread in registers.  Shared memory holds one padded tile per operand; twiddles come
// from per-axis tables w_N^e = exp(-2 pi i e/N) built in FP64.
#pragma once
#include <cuda.h>  // CUtensorMap (type only; the plan encodes maps through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <stdint.h>
#include "df32.cuh"

namespace etd {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<dfloat> { using type = dcomplex; };

// Read-only loads of twiddles and warp shuffles for each element type.
__device__ __forceinline__ float2 ldg_c(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_c(const double2* p) { return __ldg(p); }
__device__ __forceinline__ dcomplex ldg_c(const dcomplex* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return dcomplex{dfloat(v.x, v.y), dfloat(v.z, v.w)};
}
__device__ __forceinline__ float shfl(float v, int lane, int width) { return __shfl_sync(0xffffffffu, v, lane, width); }
__device__ __forceinline__ double shfl(double v, int lane, int width) { return __shfl_sync(0xffffffffu, v, lane, width); }
__device__ __forceinline__ dfloat shfl(dfloat v, int lane, int width) {
  return dfloat(__shfl_sync(0xffffffffu, v.hi, lane, width), __shfl_sync(0xffffffffu, v.lo, lane, width));
}

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return C{a.x * s, a.y * s}; }

// Grid geometry and the four-step split, passed by value to every kernel.
struct Geo {
  int dim, nx, ny, nz, nxh;
  int lx, ly;          // log2 nx, log2 ny (neighbour arithmetic of the pointwise kernels)
  int pow2;            // every extent a power of two (shift-and-mask neighbours)
  int Y1, Y2, ZB, KB;
  long long n, nhat;
  double hx, hy, hz;
};

// Launch shapes of the pass kernels (threads per CTA, CTAs per SM the FP32 register budget
// is sized for; FP64 kernels keep the full register file) and the number of z-planes per pass-A tile in FP32 (FP64 uses half).
#ifndef ETD_PASSA_THREADS
#define ETD_PASSA_THREADS 512
#endif
#ifndef ETD_PASSA_MINB
#define ETD_PASSA_MINB 2
#endif
#ifndef ETD_PASSB_THREADS
#define ETD_PASSB_THREADS 256
#endif
#ifndef ETD_PASSB_MINB
#define ETD_PASSB_MINB 2
#endif
#ifndef ETD_ZB32
#define ETD_ZB32 4
#endif

// Shared-memory padding: one spare slot every 16 complex elements (bank spreading).
__host__ __device__ __forceinline__ int pad16(int k) { return k + (k >> 4); }

// R and S of the team transform of an axis of length n: S lanes (a power of two) with R values
// each, R a multiple of S (the second stage runs R/S transforms of length S per lane).  Powers
// of two up to 256: R = min(n, 16); 96 = 24 x 4.
__host__ __device__ __forceinline__ constexpr int team_R(int n) { return n == 96 ? 24 : (n < 16 ? n : 16); }
__host__ __device__ __forceinline__ constexpr int team_S(int n) { return n / team_R(n); }
// Axis lengths the two-pass transform supports.
__host__ __device__ __forceinline__ constexpr bool fft_length_ok(int n) {
  return n == 8 || n == 16 || n == 32 || n == 64 || n == 128 || n == 256 || n == 96;
}
// The long axis (x in pass A, z in pass B) of a launch: a power of two (family 0) or 96
// (family 1); each family is its own kernel instantiation, so the 24-value registers of the
// 96-point team never weigh on the power-of-two kernels.
__host__ __device__ __forceinline__ constexpr int fft_family(int n) { return n == 96 ? 1 : 0; }

// Tile row pitches.  A team's exchange scratch (S (R + 1) values) lives in the rows it works
// on: a pair of pass-A rows, one pass-B row.
__host__ __device__ __forceinline__ int pitch_a(int nx) {
  const int p = pad16(nx / 2) + 1, need = (team_S(nx) * (team_R(nx) + 1) + 1) / 2;
  return p > need ? p : need;
}
__host__ __device__ __forceinline__ int pitch_b(int nz) {
  const int p = pad16(nz - 1) + 1, need = team_S(nz) * (team_R(nz) + 1);
  return p > need ? p : need;
}


// Tile choice shared by the plan and the allocation-free entry point.  Returns false if the
// grid is not supported.  smemA: pass-A tile; smemB1: one pass-B operand tile.
//   pass A: ZB z-planes x Y2 rows per CTA; zb_req > 0 asks for ZB (a divisor of Nz), else
//           4 (8-byte complex) or 2 (16-byte complex);
//   pass B: KB consecutive kx pencil blocks of Y1 x Nz per CTA.  A team of S lanes takes one
//           row (two in 2D), so KB Y1 is at most the block's rows; kb_req > 0 asks for KB, else
//           1 in 3D (the most CTAs) and as many as the block holds in 2D.
inline int passb_max_rows(int nz) {
  const int rpt = team_R(nz) >= 8 ? 1 : 2;
  return (ETD_PASSB_THREADS / team_S(nz)) * rpt;
}
inline bool choose_tiles(Geo& g, size_t csize, size_t& smemA, size_t& smemB1, int zb_req = 0, int kb_req = 0) {
  if (!fft_length_ok(g.nx) || !fft_length_ok(g.ny) || !(g.nz == 1 || fft_length_ok(g.nz))) return false;
  g.Y2 = g.ny < 16 ? g.ny : 16;
  g.Y1 = g.ny / g.Y2;
  if (g.Y1 > 16 || g.Y2 < 2) return false;
  const int zb = zb_req > 0 ? zb_req : (csize == 8 ? ETD_ZB32 : (ETD_ZB32 > 1 ? ETD_ZB32 / 2 : 1));
  g.ZB = g.nz == 1 ? 1 : (g.nz < zb ? g.nz : zb);
  if (g.nz % g.ZB) return false;
  const int rsa = pitch_a(g.nx);
  smemA = (size_t)g.ZB * g.Y2 * rsa * csize;
  const int rsb = pitch_b(g.nz);
  const int kbmax = passb_max_rows(g.nz) / g.Y1;
  if (kb_req > 0) {
    g.KB = kb_req;
  } else if (g.nz > 1) {
    g.KB = 1;
  } else {
    g.KB = 512 / g.Y1;
  }
  if (g.KB > g.nxh) g.KB = g.nxh;
  if (g.KB < 1 || g.KB > kbmax) return false;
  smemB1 = (size_t)g.KB * g.Y1 * rsb * csize;
  return smemA <= 200 * 1024 && 2 * smemB1 <= 200 * 1024;
}

// ---- radix kernels --------------------------------------------------------------------
template <typename C, bool INV> __device__ __forceinline__ void dft2(C* v) {
  C t = v[0];
  v[0] = cadd(t, v[1]);
  v[1] = csub(t, v[1]);
}

template <typename C, bool INV> __device__ __forceinline__ void dft4(C* v) {
  C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  C t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
  t3 = INV ? C{-t3.y, t3.x} : C{t3.y, -t3.x};  // times +i (inverse) or -i (forward)
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}

// 8-point DFT as radix 2 x 4: X[2k] = DFT4(v_r + v_{r+4}), X[2k+1] = DFT4((v_r - v_{r+4}) w8^r).
template <typename C, bool INV> __device__ __forceinline__ void dft8(C* v) {
  using T = decltype(v[0].x);
  const T s = (T)0.70710678118654752440;
  C a[4], b[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    a[r] = cadd(v[r], v[r + 4]);
    b[r] = csub(v[r], v[r + 4]);
  }
  if (INV) {
    b[1] = C{s * (b[1].x - b[1].y), s * (b[1].x + b[1].y)};
    b[2] = C{-b[2].y, b[2].x};
    b[3] = C{-s * (b[3].x + b[3].y), s * (b[3].x - b[3].y)};
  } else {
    b[1] = C{s * (b[1].x + b[1].y), s * (b[1].y - b[1].x)};
    b[2] = C{b[2].y, -b[2].x};
    b[3] = C{s * (b[3].y - b[3].x), -s * (b[3].x + b[3].y)};
  }
  dft4<C, INV>(a);
  dft4<C, INV>(b);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = a[k];
    v[2 * k + 1] = b[k];
  }
}

// 16-point DFT as 4 x 4 (inner DFT4 over n2 for each n1, twiddle w16^(n1 k1), outer DFT4).
template <typename C, bool INV> __device__ __forceinline__ void dft16(C* v) {
  using T = decltype(v[0].x);
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173, h = (T)0.70710678118654752440;
  const C w[10] = {C{1, 0}, C{c1, -s1}, C{h, -h}, C{s1, -c1}, C{0, -1}, C{-s1, -c1}, C{-h, -h}, C{-c1, -s1},
                   C{-1, 0}, C{-c1, s1}};
  C a[4][4];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) a[n1][n2] = v[n1 + 4 * n2];
    dft4<C, INV>(a[n1]);
  }
#pragma unroll
  for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) a[n1][k1] = INV ? cmulc(a[n1][k1], w[n1 * k1]) : cmul(a[n1][k1], w[n1 * k1]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft4<C, INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
  }
}

// 3-point DFT: X0 = a + b + c, X1,2 = a - (b + c)/2 -/+ i (sqrt(3)/2)(b - c) (forward).
template <typename C, bool INV> __device__ __forceinline__ void dft3(C* v) {
  using T = decltype(v[0].x);
  const T h = (T)0.5, s3 = (T)0.86602540378443864676;
  const C t1 = cadd(v[1], v[2]);
  const C t2 = C{v[0].x - h * t1.x, v[0].y - h * t1.y};
  const C d = csub(v[1], v[2]);
  const C sd = C{s3 * d.x, s3 * d.y};
  v[0] = cadd(v[0], t1);
  if (INV) {
    v[1] = C{t2.x - sd.y, t2.y + sd.x};
    v[2] = C{t2.x + sd.y, t2.y - sd.x};
  } else {
    v[1] = C{t2.x + sd.y, t2.y - sd.x};
    v[2] = C{t2.x - sd.y, t2.y + sd.x};
  }
}

template <typename C, int N, bool INV> __device__ __forceinline__ void dftN(C* v);

// N = N1 N2 point DFT by one split: Y[n1][k2] = DFT_N2 over n2 of v[n1 + N1 n2], times
// w_N^(n1 k2), then the N1-point DFT over n1 gives X[k2 + N2 k1].  w[m] = w_N^m.
template <typename C, int N1, int N2, bool INV, int NW>
__device__ __forceinline__ void dft_split(C* v, const C (&w)[NW]) {
  C a[N1][N2];
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) {
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) a[n1][n2] = v[n1 + N1 * n2];
    dftN<C, N2, INV>(a[n1]);
  }
#pragma unroll
  for (int n1 = 1; n1 < N1; ++n1)
#pragma unroll
    for (int k2 = 1; k2 < N2; ++k2) a[n1][k2] = INV ? cmulc(a[n1][k2], w[n1 * k2]) : cmul(a[n1][k2], w[n1 * k2]);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    C b[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) b[n1] = a[n1][k2];
    dftN<C, N1, INV>(b);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k2 + N2 * k1] = b[k1];
  }
}

template <typename C, bool INV> __device__ __forceinline__ void dft6(C* v) {
  using T = decltype(v[0].x);
  const C w[3] = {C{(T)1.0, (T)0.0}, C{(T)0.5, (T)-0.86602540378443864676}, C{(T)-0.5, (T)-0.86602540378443864676}};
  dft_split<C, 2, 3, INV>(v, w);
}

template <typename C, bool INV> __device__ __forceinline__ void dft12(C* v) {
  using T = decltype(v[0].x);
  const T c = (T)0.86602540378443864676, h = (T)0.5;
  const C w[7] = {C{(T)1.0, (T)0.0}, C{c, -h}, C{h, -c}, C{(T)0.0, (T)-1.0}, C{-h, -c}, C{-c, -h}, C{(T)-1.0, (T)0.0}};
  dft_split<C, 4, 3, INV>(v, w);
}

template <typename C, bool INV> __device__ __forceinline__ void dft24(C* v) {
  using T = decltype(v[0].x);
  const T a = (T)0.96592582628906828675, b = (T)0.25881904510252076235, c = (T)0.86602540378443864676,
          h = (T)0.5, r = (T)0.70710678118654752440;
  // w_24^m, m = 0..14
  const C w[15] = {C{(T)1.0, (T)0.0}, C{a, -b}, C{c, -h}, C{r, -r}, C{h, -c}, C{b, -a}, C{(T)0.0, (T)-1.0},
                   C{-b, -a}, C{-h, -c}, C{-r, -r}, C{-c, -h}, C{-a, -b}, C{(T)-1.0, (T)0.0}, C{-a, b}, C{-c, h}};
  dft_split<C, 8, 3, INV>(v, w);
}

// Natural-order DFT of compile-time length N in registers (N = 1, 2, 3, 4, 6, 8, 12, 16, 24).
template <typename C, int N, bool INV> __device__ __forceinline__ void dftN(C* v) {
  if constexpr (N == 2) dft2<C, INV>(v);
  else if constexpr (N == 3) dft3<C, INV>(v);
  else if constexpr (N == 4) dft4<C, INV>(v);
  else if constexpr (N == 6) dft6<C, INV>(v);
  else if constexpr (N == 8) dft8<C, INV>(v);
  else if constexpr (N == 12) dft12<C, INV>(v);
  else if constexpr (N == 16) dft16<C, INV>(v);
  else if constexpr (N == 24) dft24<C, INV>(v);
}


// Team FFT of length N = R * S on S lanes (lane rank t) holding R values each, R = min(N, 16).
// Lane t holds element t + S r in v[r] on entry and on exit, in both directions.  Forward:
// an R-point DFT over r in registers, the twiddle w_N^(t k1), one exchange through the team's
// shared-memory scratch (pitch R + 1: conflict-free both ways), then R/S DFTs of length S
// over the former lane index; element k1 + R k2 with k1 = t + S h lands in v[h + (R/S) k2].
// The inverse (unnormalised) is the forward transform of the conjugate, conjugated.  scr
// holds S (R + 1) values and may alias the data the lanes just loaded (the call starts with a
// warp barrier); every lane of the warp must call it, and teams without work pass act = false
// (they keep off the scratch but still take the warp barriers).
template <typename C, int R, int S, bool INV>
__device__ __forceinline__ void team_fft(C (&v)[R], int t, C* scr, const C* __restrict__ tw, bool act = true) {
  if (INV) {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r].y = -v[r].y;
  }
  dftN<C, R, false>(v);
  if (S > 1) {
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) v[k1] = cmul(v[k1], ldg_c(&tw[t * k1]));
    __syncwarp();
    if (act) {
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) scr[t * (R + 1) + k1] = v[k1];
    }
    __syncwarp();
    constexpr int H = R / S;
#pragma unroll
    for (int h = 0; h < H; ++h) {
      C u[S];
#pragma unroll
      for (int q = 0; q < S; ++q) u[q] = act ? scr[q * (R + 1) + t + S * h] : C{0, 0};
      dftN<C, S, false>(u);
#pragma unroll
      for (int k2 = 0; k2 < S; ++k2) v[h + H * k2] = u[k2];
    }
  }
  if (INV) {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r].y = -v[r].y;
  }
}

// Wavenumber bookkeeping of one spectral element.
struct Wave {
  int kx, ky, kz;   // raw spectral indices (kx < Nx/2+1)
  int fx, fy, fz;   // folded |index| (Sec. 3.2: i for i <= N/2, N - i above)
  int sx, sy, sz;   // signed index for first derivatives, 0 at the Nyquist index
  int m;            // fx^2 + fy^2 + fz^2 (the integer |k|^2 of a cubic box)
};

__device__ __forceinline__ void fold(int i, int n, int& f, int& s) {
  const int h = n >> 1;
  f = (i <= h) ? i : n - i;
  s = (i < h) ? i : (i == h ? 0 : i - n);
}

__device__ __forceinline__ Wave make_wave(const Geo& g, int kx, int ky, int kz) {
  Wave w;
  w.kx = kx;
  w.ky = ky;
  w.kz = kz;
  fold(kx, g.nx, w.fx, w.sx);
  fold(ky, g.ny, w.fy, w.sy);
  fold(kz, g.nz, w.fz, w.sz);
  w.m = w.fx * w.fx + w.fy * w.fy + w.fz * w.fz;
  return w;
}


// Inverse pass-A epilogues: epi(i, v) stores output i.  One with kSums also adds terms to
// the partial sums of a row pair (Epi::Part, live only while the pair is stored), which
// fold() moves into the thread's FP64 accumulators (Epi::Acc) and finish() sums over the
// CTA when the tile is done.
struct NoAcc {};
template <typename Epi, typename T>
__device__ __forceinline__ void epi_put(const Epi& e, long long i, T v, typename Epi::Part& part) {
  if constexpr (Epi::kSums) e(i, v, part);
  else e(i, v);
}

// Up to five output arrays of a pass-B launch, passed by value.
template <typename C> struct OutP {
  C* p[5];
};

// ---- pass A: x real-to-complex + inner y DFT ------------------------------------------
// Tile: rows r = zz * Y2 + j (plane z0 + zz, y = n1 + Y1 j), row stride pad16(nxh-1)+1.

template <typename T, typename Pro, int R, int S>
__device__ __forceinline__ void passA_rows_fwd(const Geo& g, const Pro& pro, typename Cplx<T>::type* tile, int rs,
                                               int z0, int n1, const typename Cplx<T>::type* __restrict__ twx) {
  using C = typename Cplx<T>::type;
  const int t = threadIdx.x & (S - 1);
  const int team = threadIdx.x / S, nteams = blockDim.x / S;
  const int ncrows = (g.ZB * g.Y2) >> 1;
  const int half = g.nx >> 1;
  for (int base = 0; base < ncrows; base += nteams) {
    const int q = base + team;
    const bool ok = q < ncrows;
    C v[R];
    const int r0 = 2 * q, r1 = r0 + 1;
    const long long i0 = ((long long)(z0 + r0 / g.Y2) * g.ny + n1 + g.Y1 * (r0 % g.Y2)) * g.nx;
    const long long i1 = ((long long)(z0 + r1 / g.Y2) * g.ny + n1 + g.Y1 * (r1 % g.Y2)) * g.nx;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int x = t + S * j;
      v[j] = ok ? C{pro(i0 + x), pro(i1 + x)} : C{0, 0};
    }
    // the row pair's two tile rows (2 rs >= S (R + 1) values) double as the exchange scratch
    C* row = tile + (ok ? r0 : 0) * rs;
    team_fft<C, R, S, false>(v, t, row, twx, ok);
    __syncwarp();
    // unpack the two real rows, A[k] = (Z[k] + conj Z[N-k])/2, B[k] = (Z[k] - conj Z[N-k])/(2i),
    // for k = t + S r <= N/2.  Z[N-k] sits on lane (S - t) mod S in register R-1-r (R-r mod R
    // on lane 0), fetched with one shuffle per value.
    const int pl = (S - t) & (S - 1);
#pragma unroll
    for (int r = 0; r <= R / 2; ++r) {
      const C send = (t == 0) ? v[(R - r) % R] : v[R - 1 - r];
      C zc;
      if (S > 1) {
        zc.x = shfl(send.x, pl, S);
        zc.y = shfl(send.y, pl, S);
      } else {
        zc = send;
      }
      const int k = t + S * r;
      if (ok && k <= half) {
        const C z = v[r];
        row[pad16(k)] = C{(T)0.5 * (z.x + zc.x), (T)0.5 * (z.y - zc.y)};
        row[rs + pad16(k)] = C{(T)0.5 * (z.y + zc.y), (T)0.5 * (zc.x - z.x)};
      }
    }
    __syncwarp();
  }
}

template <typename T, int Y>
__device__ __forceinline__ void passA_cols_fwd(const Geo& g, const typename Cplx<T>::type* tile, int rs, int z0,
                                               int n1, typename Cplx<T>::type* __restrict__ out,
                                               const typename Cplx<T>::type* __restrict__ twy) {
  using C = typename Cplx<T>::type;
  const int ncols = g.ZB * g.nxh;
  for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
    const int zz = col % g.ZB, kx = col / g.ZB;
    C v[Y > 1 ? Y : 1];
#pragma unroll
    for (int j = 0; j < Y; ++j) v[j] = tile[(zz * Y + j) * rs + pad16(kx)];
    dftN<C, Y, false>(v);
#pragma unroll
    for (int k2 = 0; k2 < Y; ++k2) {
      C x = v[k2];
      if (n1) x = cmul(x, ldg_c(&twy[n1 * k2]));
      out[((long long)(k2 * g.nxh + kx) * g.Y1 + n1) * g.nz + z0 + zz] = x;
    }
  }
}

// ---- TMA staging of the pass-A intermediate -------------------------------------------
// One 4-D tensor copy per CTA moves the block's part of the intermediate,
// I[k2][kx][n1][z0 .. z0+ZB) (box: 2 ZB scalars x 1 x Nx/2+1 x Y2, dense, k2 slowest),
// between shared memory and HBM: the 32-byte runs of the four-step layout are gathered or
// scattered by the copy engine instead of by 16 loads or stores per thread.  Completion of a
// load is tracked by an mbarrier; every wait is bounded and a copy that does not complete
// sets the plan's status word (7) and ends the block.
struct PassAIn {
  int tma;          // 1: stage the block's intermediate with one tensor copy; 0: plain loads/stores
  uint32_t bytes;   // bytes of one staged box
  int bar_off;      // byte offset of the mbarrier (and, forward, the leftover columns) in dynamic shared memory
  int* status;      // plan status word
  long long tries;  // polls of the copy's mbarrier before the block gives up (default 2^22)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// Store of a staged box; returns once the copy has read shared memory.
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Bounded wait for phase `parity` of the barrier: true once it completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long tries) {
  for (long long it = 0; it < tries; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Column stage of the forward into the staged box (which overlaps the tile): the leftover
// columns beyond one per thread are transformed first into a side buffer, then every thread
// reads its column into registers, and after a barrier the block writes the box.
template <typename T, int Y>
__device__ __forceinline__ void passA_cols_fwd_staged(const Geo& g, typename Cplx<T>::type* tile, int rs, int n1,
                                                      typename Cplx<T>::type* side,
                                                      const typename Cplx<T>::type* __restrict__ twy) {
  using C = typename Cplx<T>::type;
  C* stg = tile;
  const int ncols = g.ZB * g.nxh, nt = blockDim.x, t = threadIdx.x;
  const int nmain = ncols < nt ? ncols : nt, ntail = ncols - nmain;
  C v[Y > 1 ? Y : 1];
  if (t < ntail) {
    const int col = nmain + t, zz = col % g.ZB, kx = col / g.ZB;
#pragma unroll
    for (int j = 0; j < Y; ++j) v[j] = tile[(zz * Y + j) * rs + pad16(kx)];
    dftN<C, Y, false>(v);
#pragma unroll
    for (int k2 = 0; k2 < Y; ++k2) side[t * Y + k2] = (n1 && k2) ? cmul(v[k2], ldg_c(&twy[n1 * k2])) : v[k2];
  }
  const bool mine = t < nmain;
  const int zz = t % g.ZB, kx = t / g.ZB;
  if (mine) {
#pragma unroll
    for (int j = 0; j < Y; ++j) v[j] = tile[(zz * Y + j) * rs + pad16(kx)];
  }
  __syncthreads();
  if (mine) {
    dftN<C, Y, false>(v);
#pragma unroll
    for (int k2 = 0; k2 < Y; ++k2) {
      C x = v[k2];
      if (n1 && k2) x = cmul(x, ldg_c(&twy[n1 * k2]));
      stg[(k2 * g.nxh + kx) * g.ZB + zz] = x;
    }
  }
  if (t < ntail * Y) {
    const int tcol = nmain + t / Y, tk2 = t % Y;
    stg[(tk2 * g.nxh + tcol / g.ZB) * g.ZB + tcol % g.ZB] = side[t];
  }
}

template <typename T, typename Pro, int FAM = 0>
__global__ void __launch_bounds__(ETD_PASSA_THREADS, sizeof(T) == 4 ? ETD_PASSA_MINB : 1) passA_fwd(Geo g, Pro pro, typename Cplx<T>::type* __restrict__ out,
                                                 const typename Cplx<T>::type* __restrict__ twx,
                                                 const typename Cplx<T>::type* __restrict__ twy,
                                                 const __grid_constant__ CUtensorMap tout, PassAIn st) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(128) unsigned char smemA_raw[];
  C* tile = reinterpret_cast<C*>(smemA_raw);
  const int rs = pitch_a(g.nx);
  const int zb = blockIdx.x / g.Y1, n1 = blockIdx.x % g.Y1;
  const int z0 = zb * g.ZB;
  if constexpr (FAM == 1) {
    passA_rows_fwd<T, Pro, 24, 4>(g, pro, tile, rs, z0, n1, twx);
  } else {
    switch (g.nx) {
      case 8: passA_rows_fwd<T, Pro, 8, 1>(g, pro, tile, rs, z0, n1, twx); break;
      case 16: passA_rows_fwd<T, Pro, 16, 1>(g, pro, tile, rs, z0, n1, twx); break;
      case 32: passA_rows_fwd<T, Pro, 16, 2>(g, pro, tile, rs, z0, n1, twx); break;
      case 64: passA_rows_fwd<T, Pro, 16, 4>(g, pro, tile, rs, z0, n1, twx); break;
      case 128: passA_rows_fwd<T, Pro, 16, 8>(g, pro, tile, rs, z0, n1, twx); break;
      default: passA_rows_fwd<T, Pro, 16, 16>(g, pro, tile, rs, z0, n1, twx); break;
    }
  }
  __syncthreads();
  if (st.tma && (smem_u32(tile) & 127u) == 0) {
    C* side = reinterpret_cast<C*>(smemA_raw + st.bar_off + 16);
    switch (g.Y2) {
      case 2: passA_cols_fwd_staged<T, 2>(g, tile, rs, n1, side, twy); break;
      case 4: passA_cols_fwd_staged<T, 4>(g, tile, rs, n1, side, twy); break;
      case 8: passA_cols_fwd_staged<T, 8>(g, tile, rs, n1, side, twy); break;
      default: passA_cols_fwd_staged<T, 16>(g, tile, rs, n1, side, twy); break;
    }
    // the box's generic-proxy writes become visible to the copy engine, then one thread stores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) tma_store_4d(&tout, tile, 2 * z0, n1, 0, 0);
    return;
  }
  switch (g.Y2) {
    case 2: passA_cols_fwd<T, 2>(g, tile, rs, z0, n1, out, twy); break;
    case 4: passA_cols_fwd<T, 4>(g, tile, rs, z0, n1, out, twy); break;
    case 8: passA_cols_fwd<T, 8>(g, tile, rs, z0, n1, out, twy); break;
    default: passA_cols_fwd<T, 16>(g, tile, rs, z0, n1, out, twy); break;
  }
}

template <typename T, int Y>
__device__ __forceinline__ void passA_cols_inv(const Geo& g, typename Cplx<T>::type* tile, int rs, int z0, int n1,
                                               const typename Cplx<T>::type* __restrict__ in,
                                               const typename Cplx<T>::type* __restrict__ twy) {
  using C = typename Cplx<T>::type;
  const int ncols = g.ZB * g.nxh;
  for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
    const int zz = col % g.ZB, kx = col / g.ZB;
    C v[Y > 1 ? Y : 1];
#pragma unroll
    for (int k2 = 0; k2 < Y; ++k2) {
      C x = in[((long long)(k2 * g.nxh + kx) * g.Y1 + n1) * g.nz + z0 + zz];
      if (n1) x = cmulc(x, ldg_c(&twy[n1 * k2]));
      v[k2] = x;
    }
    dftN<C, Y, true>(v);
#pragma unroll
    for (int j = 0; j < Y; ++j) tile[(zz * Y + j) * rs + pad16(kx)] = v[j];
  }
}

// Column stage of the inverse from the staged box: every thread first reads its column of Y
// values (and, when ZB (Nx/2+1) exceeds the block by at most blockDim/Y columns, one value of
// a leftover column) into registers, then the whole block writes the tile over the box.
template <typename T, int Y>
__device__ __forceinline__ void passA_cols_inv_staged(const Geo& g, typename Cplx<T>::type* tile, int rs, int n1,
                                                      const typename Cplx<T>::type* __restrict__ twy) {
  using C = typename Cplx<T>::type;
  const C* stg = tile;
  const int ncols = g.ZB * g.nxh, nt = blockDim.x, t = threadIdx.x;
  const int nmain = ncols < nt ? ncols : nt, ntail = ncols - nmain;
  C v[Y > 1 ? Y : 1];
  const bool mine = t < nmain;
  const int zz = t % g.ZB, kx = t / g.ZB;
  if (mine) {
#pragma unroll
    for (int k2 = 0; k2 < Y; ++k2) v[k2] = stg[(k2 * g.nxh + kx) * g.ZB + zz];
  }
  const bool tl = t < ntail * Y;
  const int tcol = nmain + t / Y, tk2 = t % Y;
  C xt = C{0, 0};
  if (tl) xt = stg[(tk2 * g.nxh + tcol / g.ZB) * g.ZB + tcol % g.ZB];
  __syncthreads();
  if (mine) {
    if (n1) {
#pragma unroll
      for (int k2 = 1; k2 < Y; ++k2) v[k2] = cmulc(v[k2], ldg_c(&twy[n1 * k2]));
    }
    dftN<C, Y, true>(v);
#pragma unroll
    for (int j = 0; j < Y; ++j) tile[(zz * Y + j) * rs + pad16(kx)] = v[j];
  }
  if (ntail > 0) {
    if (tl) {
      if (n1) xt = cmulc(xt, ldg_c(&twy[n1 * tk2]));
      tile[((tcol % g.ZB) * Y + tk2) * rs + pad16(tcol / g.ZB)] = xt;
    }
    __syncthreads();
    if (t < ntail) {
      const int col = nmain + t, z2 = col % g.ZB, k = col / g.ZB;
#pragma unroll
      for (int k2 = 0; k2 < Y; ++k2) v[k2] = tile[(z2 * Y + k2) * rs + pad16(k)];
      dftN<C, Y, true>(v);
#pragma unroll
      for (int j = 0; j < Y; ++j) tile[(z2 * Y + j) * rs + pad16(k)] = v[j];
    }
  }
}

template <typename T, typename Epi, int R, int S>
__device__ __forceinline__ void passA_rows_inv(const Geo& g, const Epi& epi, typename Cplx<T>::type* tile, int rs,
                                               int z0, int n1, const typename Cplx<T>::type* __restrict__ twx,
                                               typename Epi::Acc& acc) {
  using C = typename Cplx<T>::type;
  const int t = threadIdx.x & (S - 1);
  const int team = threadIdx.x / S, nteams = blockDim.x / S;
  const int ncrows = (g.ZB * g.Y2) >> 1;
  const int N = g.nx, half = g.nx >> 1;
  for (int base = 0; base < ncrows; base += nteams) {
    const int q = base + team;
    const bool ok = q < ncrows;
    const int r0 = 2 * q, r1 = r0 + 1;
    C* ra = tile + (ok ? r0 : 0) * rs;
    const C* rb = ra + rs;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = t + S * r;
      C A = C{0, 0}, B = C{0, 0};
      if (ok) {
        if (k <= half) {
          A = ra[pad16(k)];
          B = rb[pad16(k)];
          if (k == 0 || k == half) {
            A.y = 0;
            B.y = 0;
          }
        } else {
          A = ra[pad16(N - k)];
          B = rb[pad16(N - k)];
          A.y = -A.y;
          B.y = -B.y;
        }
      }
      v[r] = C{A.x - B.y, A.y + B.x};
    }
    if (ok && Epi::kPrefetch) {
      const long long p0 = ((long long)(z0 + r0 / g.Y2) * g.ny + n1 + g.Y1 * (r0 % g.Y2)) * g.nx;
      const long long p1 = ((long long)(z0 + r1 / g.Y2) * g.ny + n1 + g.Y1 * (r1 % g.Y2)) * g.nx;
      const int nl = N >= 32 ? N / 32 : 1;
      for (int q = t; q < 2 * nl; q += S) epi.prefetch((q < nl ? p0 : p1) + 32 * (q % nl));
    }
    // the pair's rows, now held in registers, serve as the exchange scratch
    team_fft<C, R, S, true>(v, t, ra, twx, ok);
    if (ok) {
      const long long i0 = ((long long)(z0 + r0 / g.Y2) * g.ny + n1 + g.Y1 * (r0 % g.Y2)) * g.nx;
      const long long i1 = ((long long)(z0 + r1 / g.Y2) * g.ny + n1 + g.Y1 * (r1 % g.Y2)) * g.nx;
      typename Epi::Part part{};
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int x = t + S * j;
        epi_put(epi, i0 + x, v[j].x, part);
        epi_put(epi, i1 + x, v[j].y, part);
      }
      epi.fold(part, acc);
    }
  }
}

template <typename T, typename Epi, int FAM = 0>
__global__ void __launch_bounds__(ETD_PASSA_THREADS, sizeof(T) == 4 ? ETD_PASSA_MINB : 1) passA_inv(Geo g, const typename Cplx<T>::type* __restrict__ in, Epi epi,
                                                 const typename Cplx<T>::type* __restrict__ twx,
                                                 const typename Cplx<T>::type* __restrict__ twy,
                                                 const __grid_constant__ CUtensorMap tin, PassAIn st) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(128) unsigned char smemA_raw[];
  C* tile = reinterpret_cast<C*>(smemA_raw);
  const int rs = pitch_a(g.nx);
  const int zb = blockIdx.x / g.Y1, n1 = blockIdx.x % g.Y1;
  const int z0 = zb * g.ZB;
  // the copy's shared-memory destination must be 128-byte aligned; otherwise load directly
  if (st.tma && (smem_u32(tile) & 127u) == 0) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(smemA_raw + st.bar_off);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tma_load_4d(tile, &tin, 2 * z0, n1, 0, 0, bar, st.bytes);
    }
    const bool ok = mbar_wait(bar, 0, st.tries);
    if (__syncthreads_or(!ok)) {
      // the copy writes this block's shared memory: give it one more bounded chance to land
      // before the block leaves
      if (threadIdx.x == 0) {
        mbar_wait(bar, 0, 1LL << 22);
        atomicCAS(st.status, 0, 7);
      }
      return;
    }
    switch (g.Y2) {
      case 2: passA_cols_inv_staged<T, 2>(g, tile, rs, n1, twy); break;
      case 4: passA_cols_inv_staged<T, 4>(g, tile, rs, n1, twy); break;
      case 8: passA_cols_inv_staged<T, 8>(g, tile, rs, n1, twy); break;
      default: passA_cols_inv_staged<T, 16>(g, tile, rs, n1, twy); break;
    }
  } else {
    switch (g.Y2) {
      case 2: passA_cols_inv<T, 2>(g, tile, rs, z0, n1, in, twy); break;
      case 4: passA_cols_inv<T, 4>(g, tile, rs, z0, n1, in, twy); break;
      case 8: passA_cols_inv<T, 8>(g, tile, rs, z0, n1, in, twy); break;
      default: passA_cols_inv<T, 16>(g, tile, rs, z0, n1, in, twy); break;
    }
  }
  __syncthreads();
  typename Epi::Acc acc{};
  if constexpr (FAM == 1) {
    passA_rows_inv<T, Epi, 24, 4>(g, epi, tile, rs, z0, n1, twx, acc);
  } else {
    switch (g.nx) {
      case 8: passA_rows_inv<T, Epi, 8, 1>(g, epi, tile, rs, z0, n1, twx, acc); break;
      case 16: passA_rows_inv<T, Epi, 16, 1>(g, epi, tile, rs, z0, n1, twx, acc); break;
      case 32: passA_rows_inv<T, Epi, 16, 2>(g, epi, tile, rs, z0, n1, twx, acc); break;
      case 64: passA_rows_inv<T, Epi, 16, 4>(g, epi, tile, rs, z0, n1, twx, acc); break;
      case 128: passA_rows_inv<T, Epi, 16, 8>(g, epi, tile, rs, z0, n1, twx, acc); break;
      default: passA_rows_inv<T, Epi, 16, 16>(g, epi, tile, rs, z0, n1, twx, acc); break;
    }
  }
  epi.finish(acc);
}

// ---- pass B: outer y DFT + z FFT, spectral operator, inverse ---------------------------
// Tile rows are (kxl, k1) pairs (row index kxl * Y1 + k1) of Nz values, row stride
// pad16(Nz-1)+1.  Op supplies NI (intermediates transformed forward, 0..2),
// combine(e, global index, wave, s0, s1) on the spectra (base left in s0) and nout
// outputs out(o, base, wave), each inverse-transformed into outs.p[o].

template <typename T, int Y, bool INV>
__device__ __forceinline__ void passB_cols(const Geo& g, int kbn, const typename Cplx<T>::type* src,
                                           long long cb, typename Cplx<T>::type* tile, int rs,
                                           typename Cplx<T>::type* dst) {
  using C = typename Cplx<T>::type;
  const int ncols = kbn * g.nz;
  for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
    const int kxl = col / g.nz, z = col - kxl * g.nz;
    C v[Y > 1 ? Y : 1];
    if (!INV) {
#pragma unroll
      for (int n1 = 0; n1 < Y; ++n1) v[n1] = src[cb + (long long)(kxl * Y + n1) * g.nz + z];
      dftN<C, Y, false>(v);
#pragma unroll
      for (int k1 = 0; k1 < Y; ++k1) tile[(kxl * Y + k1) * rs + pad16(z)] = v[k1];
    } else {
#pragma unroll
      for (int k1 = 0; k1 < Y; ++k1) v[k1] = tile[(kxl * Y + k1) * rs + pad16(z)];
      dftN<C, Y, true>(v);
#pragma unroll
      for (int n1 = 0; n1 < Y; ++n1) dst[cb + (long long)(kxl * Y + n1) * g.nz + z] = v[n1];
    }
  }
}

// Forward column stage of two inputs at once: both columns' loads are in flight together.
template <typename T, int Y>
__device__ __forceinline__ void passB_cols2(const Geo& g, int kbn, const typename Cplx<T>::type* src0,
                                            const typename Cplx<T>::type* src1, long long cb,
                                            typename Cplx<T>::type* tile0, typename Cplx<T>::type* tile1, int rs) {
  using C = typename Cplx<T>::type;
  const int ncols = kbn * g.nz;
  for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
    const int kxl = col / g.nz, z = col - kxl * g.nz;
    C v[Y > 1 ? Y : 1], w[Y > 1 ? Y : 1];
#pragma unroll
    for (int n1 = 0; n1 < Y; ++n1) {
      v[n1] = src0[cb + (long long)(kxl * Y + n1) * g.nz + z];
      w[n1] = src1[cb + (long long)(kxl * Y + n1) * g.nz + z];
    }
    dftN<C, Y, false>(v);
    dftN<C, Y, false>(w);
#pragma unroll
    for (int k1 = 0; k1 < Y; ++k1) {
      tile0[(kxl * Y + k1) * rs + pad16(z)] = v[k1];
      tile1[(kxl * Y + k1) * rs + pad16(z)] = w[k1];
    }
  }
}

template <typename T, bool INV>
__device__ __forceinline__ void passB_cols_any(const Geo& g, int kbn, const typename Cplx<T>::type* src, long long cb,
                                               typename Cplx<T>::type* tile, int rs, typename Cplx<T>::type* dst) {
  switch (g.Y1) {
    case 1: passB_cols<T, 1, INV>(g, kbn, src, cb, tile, rs, dst); break;
    case 2: passB_cols<T, 2, INV>(g, kbn, src, cb, tile, rs, dst); break;
    case 4: passB_cols<T, 4, INV>(g, kbn, src, cb, tile, rs, dst); break;
    case 8: passB_cols<T, 8, INV>(g, kbn, src, cb, tile, rs, dst); break;
    case 6: passB_cols<T, 6, INV>(g, kbn, src, cb, tile, rs, dst); break;
    default: passB_cols<T, 16, INV>(g, kbn, src, cb, tile, rs, dst); break;
  }
}

template <typename T, typename Op, int R, int S>
__device__ __forceinline__ void passB_rows(const Geo& g, const Op& op, int kx0, int k2, int kbn, long long cb,
                                           typename Cplx<T>::type* tile0, typename Cplx<T>::type* tile1, int rs,
                                           OutP<typename Cplx<T>::type> outs,
                                           const typename Cplx<T>::type* __restrict__ twz) {
  using C = typename Cplx<T>::type;
  // rows per team: one for z transforms of 8 points or more (16 rows of a 3D tile over at
  // least 16 teams); two for the 2D tile (512 rows, 256 single-lane teams)
  constexpr int RPT = R >= 8 ? 1 : 2;
  const int t = threadIdx.x & (S - 1);
  const int team = threadIdx.x / S, nteams = blockDim.x / S;
  const int nrows = kbn * g.Y1;
  // spectra kept in registers across the outputs
  C base[RPT][R];
  int rowid[RPT];
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr) {
    const int row = team + rr * nteams;
    rowid[rr] = row;
    const bool ok = row < nrows;
    C* r0 = tile0 + (ok ? row : 0) * rs;
    C* r1 = tile1 + (ok ? row : 0) * rs;
    C s0[R], s1[R];
    if (Op::NI >= 1) {
#pragma unroll
      for (int j = 0; j < R; ++j) s0[j] = ok ? r0[pad16(t + S * j)] : C{0, 0};
      team_fft<C, R, S, false>(s0, t, r0, twz, ok);
    }
    if (Op::NI >= 2) {
#pragma unroll
      for (int j = 0; j < R; ++j) s1[j] = ok ? r1[pad16(t + S * j)] : C{0, 0};
      team_fft<C, R, S, false>(s1, t, r1, twz, ok);
    }
    if (ok) {
      const int kxl = row / g.Y1, k1 = row - kxl * g.Y1;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const int kz = t + S * k;
        const Wave w = make_wave(g, kx0 + kxl, k2 + g.Y2 * k1, kz);
        const int e = row * g.nz + kz;
        op.combine(e, cb + e, w, s0[k], s1[k]);
        base[rr][k] = s0[k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < R; ++k) base[rr][k] = C{0, 0};
    }
  }
  __syncthreads();
  // Outputs alternate between the two tiles, so that the row stage of output o+1 (writing
  // one tile) may run while other threads still read the other tile in the column stage of
  // output o: one block barrier per output.
  for (int o = 0; o < op.nout; ++o) {
    C* tb = (o & 1) ? tile1 : tile0;
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int row = rowid[rr];
      const bool ok = row < nrows;
      C v[R];
      const int kxl = ok ? row / g.Y1 : 0, k1 = ok ? row - kxl * g.Y1 : 0;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const int kz = t + S * k;
        v[k] = ok ? op.out(o, base[rr][k], make_wave(g, kx0 + kxl, k2 + g.Y2 * k1, kz)) : C{0, 0};
      }
      C* r0 = tb + (ok ? row : 0) * rs;
      team_fft<C, R, S, true>(v, t, r0, twz, ok);
      __syncwarp();
      if (ok) {
#pragma unroll
        for (int j = 0; j < R; ++j) r0[pad16(t + S * j)] = v[j];
      }
    }
    __syncthreads();
    passB_cols_any<T, true>(g, kbn, nullptr, cb, tb, rs, outs.p[o]);
  }
}

template <typename T, typename Op, int FAM = 0>
__global__ void __launch_bounds__(ETD_PASSB_THREADS, sizeof(T) == 4 ? ETD_PASSB_MINB : 1) passB(Geo g, Op op, const typename Cplx<T>::type* __restrict__ in0,
                                             const typename Cplx<T>::type* __restrict__ in1,
                                             OutP<typename Cplx<T>::type> outs,
                                             const typename Cplx<T>::type* __restrict__ twy,
                                             const typename Cplx<T>::type* __restrict__ twz) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rs = pitch_b(g.nz);
  const int kb = blockIdx.x / g.Y2, k2 = blockIdx.x % g.Y2;
  const int kx0 = kb * g.KB;
  const int kbn = min(g.KB, g.nxh - kx0);
  const long long cb = ((long long)(k2 * g.nxh + kx0) * g.Y1) * g.nz;
  C* tile0 = reinterpret_cast<C*>(smem_raw);
  C* tile1 = tile0 + (size_t)g.KB * g.Y1 * rs;
  // the operator's stored-spectrum reads (after the forward transforms) find their lines in L2
  if (const void* pre = op.pre()) {
    const size_t es = op.pre_elem();
    const int nl = (int)((size_t)kbn * g.Y1 * g.nz * es / 128);
    const char* base = reinterpret_cast<const char*>(pre) + (size_t)cb * es;
    for (int q = threadIdx.x; q < nl; q += blockDim.x)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(base + 128 * (size_t)q));
  }
  if (Op::NI == 2 && g.Y1 == 16) {
    passB_cols2<T, 16>(g, kbn, in0, in1, cb, tile0, tile1, rs);
  } else {
    if (Op::NI >= 1) passB_cols_any<T, false>(g, kbn, in0, cb, tile0, rs, nullptr);
    if (Op::NI >= 2) passB_cols_any<T, false>(g, kbn, in1, cb, tile1, rs, nullptr);
  }
  __syncthreads();
  if constexpr (FAM == 1) {
    passB_rows<T, Op, 24, 4>(g, op, kx0, k2, kbn, cb, tile0, tile1, rs, outs, twz);
    return;
  }
  switch (g.nz) {
    case 1: passB_rows<T, Op, 1, 1>(g, op, kx0, k2, kbn, cb, tile0, tile1, rs, outs, twz); break;
    case 8: passB_rows<T, Op, 8, 1>(g, op, kx0, k2, kbn, cb, tile0, tile1, rs, outs, twz); break;
    case 16: passB_rows<T, Op, 16, 1>(g, op, kx0, k2, kbn, cb, tile0, tile1, rs, outs, twz); break;
    case 32: passB_rows<T, Op, 16, 2>(g, op, kx0, k2, kbn, cb, tile0, tile1, rs, outs, twz); break;
    case 64: passB_rows<T, Op, 16, 4>(g, op, kx0, k2, kbn, cb, tile0, tile1, rs, outs, twz); break;
    case 128: passB_rows<T, Op, 16, 8>(g, op, kx0, k2, kbn, cb, tile0, tile1, rs, outs, twz); break;
    default: passB_rows<T, Op, 16, 16>(g, op, kx0, k2, kbn, cb, tile0, tile1, rs, outs, twz); break;
  }
}

}  // namespace etd
