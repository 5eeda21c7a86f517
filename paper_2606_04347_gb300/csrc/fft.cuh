// fft.cuh -- 2D/3D real-to-complex FFT for sm_103a in two HBM passes.
//
// Transform convention (the spectral collocation of Sec. 3.2): forward
//   F_k = sum_j f_j exp(-2 pi i j.k / N), inverse with +i and 1/N.
//
// Decomposition ("four-step" split of the y axis, Ny = Y1 * Y2, y = n1 + Y1 * n2,
// ky = k2 + Y2 * k1):
//   pass A (one CTA per z-block of ZB planes and residue n1): the Y2 rows y = n1 + Y1*j of
//     each plane are real-to-complex transformed along x (two real rows packed into one
//     complex row), then Y2-point DFTs across the rows give k2, then the twiddle
//     w_Ny^(n1 k2).  Out: intermediate I[k2][kx][n1][z].
//   pass B (one CTA per kx-block and k2): the Y1-point DFT over n1 gives k1, the Nz-point
//     DFT over z gives kz.  The spectrum sits in smem; a pointwise spectral operator runs
//     there (the ETD update), and the results go straight back through the inverse pass B.
// The spectral layout is therefore S[k2][kx][k1][kz] (complex), the same index map as the
// intermediate, so stored spectra are read and written by pass B in contiguous chunks.
//
// In shared memory every 1D transform is a batched Stockham autosort FFT (radix 8/4/2,
// ping-pong between two buffers, one barrier per stage), the formulation of Govindaraju et
// al., "High performance discrete Fourier transforms on graphics processors" (SC 2008).
// Twiddles come from per-axis FP64-built tables w_N^e = exp(-2 pi i e/N), e < N.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace etd {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

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
  int Y1, Y2, ZB, KB;
  long long n, nhat;
  double hx, hy, hz;
};

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

template <typename C, int R, bool INV> __device__ __forceinline__ void dftR(C* v) {
  if (R == 2) dft2<C, INV>(v);
  else if (R == 4) dft4<C, INV>(v);
  else dft8<C, INV>(v);
}

// One Stockham stage: `nbatch` transforms of length L, current span Ns.  Element i of
// transform b lives at base(b) + i*es, base(b) = (b / nb_in) * bs_out + (b % nb_in) * bs_in.
// batch_fast chooses which index varies fastest across threads (bank-conflict control).
template <typename C, int R, bool INV>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ src, C* __restrict__ dst, int L,
                                               int Ns, int nbatch, int nb_in, int bs_in, int bs_out,
                                               int es, const C* __restrict__ tw, int twstride,
                                               bool batch_fast) {
  const int nbf = L / R;
  const int total = nbatch * nbf;
  const int tstep = (L / (Ns * R)) * twstride;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    int b, j;
    if (batch_fast) {
      b = w % nbatch;
      j = w / nbatch;
    } else {
      j = w % nbf;
      b = w / nbf;
    }
    const int base = (b / nb_in) * bs_out + (b % nb_in) * bs_in;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[base + (j + r * nbf) * es];
    const int k = j & (Ns - 1);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C t = __ldg(&tw[r * k * tstep]);
        v[r] = INV ? cmulc(v[r], t) : cmul(v[r], t);
      }
    }
    dftR<C, R, INV>(v);
    const int ob = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[base + (ob + r * Ns) * es] = v[r];
  }
}

// Batched in-smem FFT of length L (a power of two); returns the buffer holding the result
// (a or b).  Contains __syncthreads(): every thread of the block must call it.
template <typename C, bool INV>
__device__ C* smem_fft(C* a, C* b, int L, int nbatch, int nb_in, int bs_in, int bs_out, int es,
                       const C* __restrict__ tw, int twstride, bool batch_fast) {
  C* src = a;
  C* dst = b;
  int Ns = 1;
  while (Ns < L) {
    const int rem = L / Ns;
    const int R = (rem == 16) ? 4 : (rem >= 8 ? 8 : rem);
    if (R == 8)
      stockham_stage<C, 8, INV>(src, dst, L, Ns, nbatch, nb_in, bs_in, bs_out, es, tw, twstride, batch_fast);
    else if (R == 4)
      stockham_stage<C, 4, INV>(src, dst, L, Ns, nbatch, nb_in, bs_in, bs_out, es, tw, twstride, batch_fast);
    else
      stockham_stage<C, 2, INV>(src, dst, L, Ns, nbatch, nb_in, bs_in, bs_out, es, tw, twstride, batch_fast);
    __syncthreads();
    C* t = src;
    src = dst;
    dst = t;
    Ns *= R;
  }
  return src;
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

// ---- pass A: x real-to-complex + inner y DFT ------------------------------------------
// smem: two buffers of ZB*Y2*nxh complex.
template <typename T, typename Pro>
__global__ void __launch_bounds__(512) passA_fwd(Geo g, Pro pro, typename Cplx<T>::type* __restrict__ out,
                                                 const typename Cplx<T>::type* __restrict__ twx,
                                                 const typename Cplx<T>::type* __restrict__ twy) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrows = g.ZB * g.Y2;
  const int tc = nrows * g.nxh;
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + tc;
  const int zb = blockIdx.x / g.Y1, n1 = blockIdx.x % g.Y1;
  const int z0 = zb * g.ZB;
  const int npairs = nrows >> 1;
  for (int e = threadIdx.x; e < npairs * g.nx; e += blockDim.x) {
    const int q = e / g.nx, x = e - q * g.nx;
    const int r0 = 2 * q, r1 = r0 + 1;
    const long long i0 = ((long long)(z0 + r0 / g.Y2) * g.ny + n1 + g.Y1 * (r0 % g.Y2)) * g.nx + x;
    const long long i1 = ((long long)(z0 + r1 / g.Y2) * g.ny + n1 + g.Y1 * (r1 % g.Y2)) * g.nx + x;
    bufA[e] = C{pro(i0), pro(i1)};
  }
  __syncthreads();
  C* res = smem_fft<C, false>(bufA, bufB, g.nx, npairs, npairs, g.nx, 0, 1, twx, 1, false);
  C* oth = (res == bufA) ? bufB : bufA;
  const int mask = g.nx - 1;
  for (int e = threadIdx.x; e < npairs * g.nxh; e += blockDim.x) {
    const int q = e / g.nxh, k = e - q * g.nxh;
    const C a = res[q * g.nx + k];
    const C b = res[q * g.nx + ((g.nx - k) & mask)];
    oth[(2 * q) * g.nxh + k] = C{(T)0.5 * (a.x + b.x), (T)0.5 * (a.y - b.y)};
    oth[(2 * q + 1) * g.nxh + k] = C{(T)0.5 * (a.y + b.y), (T)0.5 * (b.x - a.x)};
  }
  __syncthreads();
  C* r2 = smem_fft<C, false>(oth, res, g.Y2, g.ZB * g.nxh, g.nxh, 1, g.Y2 * g.nxh, g.nxh, twy, g.Y1, true);
  for (int e = threadIdx.x; e < tc; e += blockDim.x) {
    const int zz = e % g.ZB;
    const int t = e / g.ZB;
    const int kx = t % g.nxh, k2 = t / g.nxh;
    C v = r2[(zz * g.Y2 + k2) * g.nxh + kx];
    if (n1) v = cmul(v, __ldg(&twy[n1 * k2]));
    out[((long long)(k2 * g.nxh + kx) * g.Y1 + n1) * g.nz + z0 + zz] = v;
  }
}

template <typename T, typename Epi>
__global__ void __launch_bounds__(512) passA_inv(Geo g, const typename Cplx<T>::type* __restrict__ in, Epi epi,
                                                 const typename Cplx<T>::type* __restrict__ twx,
                                                 const typename Cplx<T>::type* __restrict__ twy) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrows = g.ZB * g.Y2;
  const int tc = nrows * g.nxh;
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + tc;
  const int zb = blockIdx.x / g.Y1, n1 = blockIdx.x % g.Y1;
  const int z0 = zb * g.ZB;
  for (int e = threadIdx.x; e < tc; e += blockDim.x) {
    const int zz = e % g.ZB;
    const int t = e / g.ZB;
    const int kx = t % g.nxh, k2 = t / g.nxh;
    C v = in[((long long)(k2 * g.nxh + kx) * g.Y1 + n1) * g.nz + z0 + zz];
    if (n1) v = cmulc(v, __ldg(&twy[n1 * k2]));
    bufA[(zz * g.Y2 + k2) * g.nxh + kx] = v;
  }
  __syncthreads();
  C* res = smem_fft<C, true>(bufA, bufB, g.Y2, g.ZB * g.nxh, g.nxh, 1, g.Y2 * g.nxh, g.nxh, twy, g.Y1, true);
  C* oth = (res == bufA) ? bufB : bufA;
  const int npairs = nrows >> 1;
  const int h = g.nx >> 1;
  for (int e = threadIdx.x; e < npairs * g.nx; e += blockDim.x) {
    const int q = e / g.nx, k = e - q * g.nx;
    C A, B;
    if (k <= h) {
      A = res[(2 * q) * g.nxh + k];
      B = res[(2 * q + 1) * g.nxh + k];
      if (k == 0 || k == h) {
        A.y = 0;
        B.y = 0;
      }
    } else {
      A = res[(2 * q) * g.nxh + g.nx - k];
      B = res[(2 * q + 1) * g.nxh + g.nx - k];
      A.y = -A.y;
      B.y = -B.y;
    }
    oth[e] = C{A.x - B.y, A.y + B.x};
  }
  __syncthreads();
  C* r2 = smem_fft<C, true>(oth, res, g.nx, npairs, npairs, g.nx, 0, 1, twx, 1, false);
  for (int e = threadIdx.x; e < npairs * g.nx; e += blockDim.x) {
    const int q = e / g.nx, x = e - q * g.nx;
    const int r0 = 2 * q, r1 = r0 + 1;
    const long long i0 = ((long long)(z0 + r0 / g.Y2) * g.ny + n1 + g.Y1 * (r0 % g.Y2)) * g.nx + x;
    const long long i1 = ((long long)(z0 + r1 / g.Y2) * g.ny + n1 + g.Y1 * (r1 % g.Y2)) * g.nx + x;
    const C v = r2[e];
    epi(i0, v.x);
    epi(i1, v.y);
  }
}

// Up to five output arrays of a pass-B launch, passed by value.
template <typename C> struct OutP {
  C* p[5];
};

// ---- pass B: outer y DFT + z FFT, spectral operator, inverse ---------------------------
// smem: three buffers of KB*Y1*nz complex.  Op supplies NI (intermediates to transform
// forward, 0..2), combine(e, global index, wave, s0, s1) run elementwise on the spectra
// (base result left in s0), nout outputs out(o, base, wave) inverse-transformed to outs[o].
template <typename C>
__device__ __forceinline__ C* passB_forward(const Geo& g, C* a, C* b, int kbn, const C* twy, const C* twz) {
  C* r = smem_fft<C, false>(a, b, g.Y1, kbn * g.nz, g.nz, 1, g.Y1 * g.nz, g.nz, twy, g.Y2, true);
  C* o = (r == a) ? b : a;
  return smem_fft<C, false>(r, o, g.nz, kbn * g.Y1, kbn * g.Y1, g.nz, 0, 1, twz, 1, false);
}

template <typename C>
__device__ __forceinline__ C* passB_inverse(const Geo& g, C* a, C* b, int kbn, const C* twy, const C* twz) {
  C* r = smem_fft<C, true>(a, b, g.nz, kbn * g.Y1, kbn * g.Y1, g.nz, 0, 1, twz, 1, false);
  C* o = (r == a) ? b : a;
  return smem_fft<C, true>(r, o, g.Y1, kbn * g.nz, g.nz, 1, g.Y1 * g.nz, g.nz, twy, g.Y2, true);
}

template <typename T, typename Op>
__global__ void __launch_bounds__(512) passB(Geo g, Op op, const typename Cplx<T>::type* __restrict__ in0,
                                             const typename Cplx<T>::type* __restrict__ in1,
                                             OutP<typename Cplx<T>::type> outs,
                                             const typename Cplx<T>::type* __restrict__ twy,
                                             const typename Cplx<T>::type* __restrict__ twz) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int slot = g.KB * g.Y1 * g.nz;
  C* buf[3] = {reinterpret_cast<C*>(smem_raw), reinterpret_cast<C*>(smem_raw) + slot,
               reinterpret_cast<C*>(smem_raw) + 2 * slot};
  const int kb = blockIdx.x / g.Y2, k2 = blockIdx.x % g.Y2;
  const int kx0 = kb * g.KB;
  const int kbn = min(g.KB, g.nxh - kx0);
  const int cl = kbn * g.Y1 * g.nz;
  const long long cb = ((long long)(k2 * g.nxh + kx0) * g.Y1) * g.nz;
  C* s0 = buf[0];
  C* s1 = buf[1];
  C* fr = buf[2];
  if (Op::NI >= 1) {
    for (int e = threadIdx.x; e < cl; e += blockDim.x) s0[e] = in0[cb + e];
    __syncthreads();
    C* r = passB_forward<C>(g, s0, fr, kbn, twy, twz);
    if (r != s0) {
      fr = s0;
      s0 = r;
    }
  }
  if (Op::NI >= 2) {
    for (int e = threadIdx.x; e < cl; e += blockDim.x) s1[e] = in1[cb + e];
    __syncthreads();
    C* r = passB_forward<C>(g, s1, fr, kbn, twy, twz);
    if (r != s1) {
      fr = s1;
      s1 = r;
    }
  }
  const int per_kx = g.Y1 * g.nz;
  for (int e = threadIdx.x; e < cl; e += blockDim.x) {
    const int kxl = e / per_kx;
    const int rem = e - kxl * per_kx;
    const int k1 = rem / g.nz, kz = rem - k1 * g.nz;
    const Wave w = make_wave(g, kx0 + kxl, k2 + g.Y2 * k1, kz);
    op.combine(e, cb + e, w, s0[e], s1[e]);
  }
  __syncthreads();
  for (int o = 0; o < op.nout; ++o) {
    C* t = s1;
    for (int e = threadIdx.x; e < cl; e += blockDim.x) {
      const int kxl = e / per_kx;
      const int rem = e - kxl * per_kx;
      const int k1 = rem / g.nz, kz = rem - k1 * g.nz;
      const Wave w = make_wave(g, kx0 + kxl, k2 + g.Y2 * k1, kz);
      t[e] = op.out(o, s0[e], w);
    }
    __syncthreads();
    C* r = passB_inverse<C>(g, t, fr, kbn, twy, twz);
    C* dst = outs.p[o];
    for (int e = threadIdx.x; e < cl; e += blockDim.x) dst[cb + e] = r[e];
    __syncthreads();
  }
}

}  // namespace etd
