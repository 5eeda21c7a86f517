// kernels.cuh -- pointwise terms, finite-difference band terms, band compaction, the band
// conjugate-gradient solve and FP64 reductions of the ETD membrane step.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include "fft.cuh"

namespace etd {

// Model coefficients in the working precision (Eq. (1.1)-(1.2), Sec. 3.1) plus grid factors.
template <typename T> struct ModelC {
  T eps_phi, eps_u, mu, lambda_surf, kappa, lambda_line, M_area, alpha, u0;
  T gamma, M, ubar, A1, A2, B1, B2, band_hi, delta, tau;
  T ih2[3];    // 1/h_d^2
  T i2h[3];    // 1/(2 h_d)
  int dim;
  int linear_only;
};

// Slots of the FP64 scalar array shared by the kernels of one plan.
enum Scal {
  S_VOL = 0,      // sum phi (current phi-stage argument)
  S_MASS = 1,     // sum G (u - ubar)  or  sum G (f(u) - ubar)
  S_GRAD = 2, S_WELL = 3, S_NONLOC = 4, S_MASSF = 5, S_VOLE = 6,
  S_MAXB = 7, S_UMIN = 8, S_UMAX = 9,
  S_A0 = 12,      // A0 itself (not a sum); set once
  S_COUNT = 16
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum added atomically to *dst (one atomic per block).  All threads call it.
__device__ __forceinline__ void block_add(double v, double* dst) {
  __shared__ double ws[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double t = (lane < nw) ? ws[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) atomicAdd(dst, t);
  }
}

__device__ __forceinline__ void atomic_max_nonneg(double* dst, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_d(double* dst, double v) {
  unsigned long long* a = reinterpret_cast<unsigned long long*>(dst);
  unsigned long long old = *a, assumed;
  do {
    assumed = old;
    if (__longlong_as_double((long long)assumed) <= v) break;
    old = atomicCAS(a, assumed, (unsigned long long)__double_as_longlong(v));
  } while (assumed != old);
}
__device__ __forceinline__ void atomic_max_d(double* dst, double v) {
  unsigned long long* a = reinterpret_cast<unsigned long long*>(dst);
  unsigned long long old = *a, assumed;
  do {
    assumed = old;
    if (__longlong_as_double((long long)assumed) >= v) break;
    old = atomicCAS(a, assumed, (unsigned long long)__double_as_longlong(v));
  } while (assumed != old);
}

// Periodic neighbours of flat index p: shifts and masks when every extent is a power of two,
// integer division otherwise.
struct Nb {
  int c, xm, xp, ym, yp, zm, zp;
};
__device__ __forceinline__ Nb neighbours(const Geo& g, int p) {
  if (!g.pow2) {
    const int x = p % g.nx, t = p / g.nx, y = t % g.ny, z = t / g.ny;
    const int sxy = g.nx * g.ny;
    const int rowbase = p - x, planebase = z * sxy, inplane = p - planebase;
    Nb n;
    n.c = p;
    n.xm = rowbase + (x == 0 ? g.nx - 1 : x - 1);
    n.xp = rowbase + (x == g.nx - 1 ? 0 : x + 1);
    n.ym = planebase + (y == 0 ? g.ny - 1 : y - 1) * g.nx + x;
    n.yp = planebase + (y == g.ny - 1 ? 0 : y + 1) * g.nx + x;
    n.zm = (z == 0 ? g.nz - 1 : z - 1) * sxy + inplane;
    n.zp = (z == g.nz - 1 ? 0 : z + 1) * sxy + inplane;
    return n;
  }
  const int mx = g.nx - 1, my = g.ny - 1, mz = g.nz - 1;
  const int sp = g.lx + g.ly;
  const int x = p & mx;
  const int y = (p >> g.lx) & my;
  const int z = p >> sp;
  const int rowbase = p - x;
  const int inplane = p & ((1 << sp) - 1);
  const int planebase = p - inplane;
  Nb n;
  n.c = p;
  n.xm = rowbase + ((x - 1) & mx);
  n.xp = rowbase + ((x + 1) & mx);
  n.ym = planebase + ((((y - 1) & my)) << g.lx) + x;
  n.yp = planebase + ((((y + 1) & my)) << g.lx) + x;
  n.zm = (((z - 1) & mz) << sp) + inplane;
  n.zp = (((z + 1) & mz) << sp) + inplane;
  return n;
}

template <typename T> __device__ __forceinline__ T gloc(T f) {  // g = 18 (f^2 - f)^2
  const T a = f * f - f;
  return (T)18 * a * a;
}
template <typename T> __device__ __forceinline__ T dW(T s) { return (T)36 * s * (s - (T)1) * ((T)2 * s - (T)1); }
template <typename T> __device__ __forceinline__ T d2W(T s) { return (T)36 * ((T)6 * s * s - (T)6 * s + (T)1); }
template <typename T> __device__ __forceinline__ T Wpot(T s) {
  const T a = s * s - s;
  return (T)18 * a * a;
}
template <typename T> __device__ __forceinline__ T find(T u) { return (T)3 * u * u - (T)2 * u * u * u; }
template <typename T> __device__ __forceinline__ T dfind(T u) { return (T)6 * u * ((T)1 - u); }
template <typename T> __device__ __forceinline__ bool in_band(T phi, T hi) {
  return fabs((T)2 * phi - (T)1) < hi;
}

// Delta_{S,h} u at p with face-averaged g (Eq. (2.3)); g evaluated from values gc, g-neighbours.
template <typename T>
__device__ __forceinline__ T surf_lap(const Geo& g, const ModelC<T>& mc, const Nb& n, const T* __restrict__ u,
                                      T gc, T gxm, T gxp, T gym, T gyp, T gzm, T gzp) {
  const T uc = u[n.c];
  T s = (((T)0.5 * (gxp + gc)) * (u[n.xp] - uc) - ((T)0.5 * (gc + gxm)) * (uc - u[n.xm])) * mc.ih2[0] +
        (((T)0.5 * (gyp + gc)) * (u[n.yp] - uc) - ((T)0.5 * (gc + gym)) * (uc - u[n.ym])) * mc.ih2[1];
  if (g.nz > 1)
    s += (((T)0.5 * (gzp + gc)) * (u[n.zp] - uc) - ((T)0.5 * (gc + gzm)) * (uc - u[n.zm])) * mc.ih2[2];
  return s;
}

// ---- pass-A prologues / epilogues ------------------------------------------------------
template <typename T> struct ProLoad {
  const T* a;
  __device__ T operator()(long long i) const { return a[i]; }
};
template <typename T> struct ProMul {
  const T* a;
  const T* b;
  __device__ T operator()(long long i) const { return a[i] * b[i]; }
};
template <typename T> struct EpiStore {
  static constexpr bool kPrefetch = false, kSums = false;
  using Acc = NoAcc;
  using Part = NoAcc;
  __device__ void prefetch(long long) const {}
  __device__ void fold(Part&, Acc&) const {}
  __device__ void finish(Acc&) const {}
  T* out;
  __device__ void operator()(long long i, T v) const { out[i] = v; }
};
// U = GU/G where G > delta, GU elsewhere (Sec. 3.3, recovery after Algorithm 1).
// u from the increment of G u over a stage: the inverse transform delivers
// d = GU_new - G u_base, and on the recovery set {G > delta} u = GU_new / G is formed as
// u_base + d / G (equal in exact arithmetic; the FP32 transform error then scales with the
// increment instead of with G u itself), elsewhere u = GU_new = G u_base + d (Algorithm 1).
__device__ __forceinline__ float div_inc(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_inc(double a, double b) { return a / b; }

// Epilogues with inputs of their own (EpiRecover) prefetch their cache lines into L2 before
// the inverse x transform of a row pair, so the loads after it find them on chip.
template <typename T> struct EpiRecover {
  static constexpr bool kPrefetch = true, kSums = false;
  using Acc = NoAcc;
  using Part = NoAcc;
  __device__ void fold(Part&, Acc&) const {}
  __device__ void finish(Acc&) const {}
  __device__ void prefetch(long long i) const {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(G + i));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(base + i));
  }
  T* out;
  const T* G;
  const T* base;
  T delta;
  __device__ void operator()(long long i, T v) const {
    const T gg = G[i];
    const T ub = base[i];
    // the quotient only forms the increment d / G, so the 2-ulp fast division suffices in FP32
    out[i] = gg > delta ? ub + div_inc(v, gg) : gg * ub + v;
  }
};
// phi^{n+1} and G^{n+1} = 18 (phi^2 - phi)^2 (Algorithm 1).
template <typename T> struct EpiPhiG {
  static constexpr bool kPrefetch = false, kSums = false;
  using Acc = NoAcc;
  using Part = NoAcc;
  __device__ void prefetch(long long) const {}
  __device__ void fold(Part&, Acc&) const {}
  __device__ void finish(Acc&) const {}
  T* phi;
  T* G;
  T* zero;   // optional: a field cleared in the same pass (the band-list R2 fills its band later)
  __device__ void operator()(long long i, T v) const {
    phi[i] = v;
    G[i] = gloc(v);
    if (zero) zero[i] = 0;
  }
};

// ---- pointwise / band kernels ----------------------------------------------------------

// R1 without its Laplacian term (Sec. 3.1), and W'(phi) - A1 phi whose spectrum receives
// kappa/(mu eps^2) lambda in pass B.  Delta phi and grad phi are spectral (pass-A outputs).
template <typename T>
__global__ void k_r1(Geo g, ModelC<T> mc, const T* __restrict__ phi, const T* __restrict__ lap,
                     const T* __restrict__ gx, const T* __restrict__ gy, const T* __restrict__ gz,
                     const T* __restrict__ u, const double* __restrict__ scal, double hvol,
                     T* __restrict__ out_rest, T* __restrict__ out_wm) {
  const T e = mc.eps_phi, e2 = e * e;
  const T dvol = (T)(hvol * scal[S_VOL] - scal[S_A0]);
  const T c_a = mc.kappa / (mc.mu * e2);
  const T c_b = mc.kappa / (mc.mu * e2 * e2);
  const T c_c = mc.lambda_surf / (mc.mu * e2);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < (int)g.n; p += gridDim.x * blockDim.x) {
    if (mc.linear_only) {
      out_rest[p] = 0;
      out_wm[p] = 0;
      continue;
    }
    const T f = phi[p], L = lap[p];
    const T ax = gx[p], ay = gy[p], az = g.nz > 1 ? gz[p] : (T)0;
    const T gn = sqrt(ax * ax + ay * ay + az * az);
    const T Wp = dW(f), Wpp = d2W(f);
    const T Wm = Wp - mc.A1 * f;
    const T uu = u[p];
    T r = c_a * (Wpp - mc.A2) * (L - mc.A1 * f / e2) - (c_b * Wpp + c_c) * Wm;
    if (in_band(f, mc.band_hi)) {
      // line-tension term with Delta_{S,h} u (g = g(phi) at the faces), band points only
      const Nb n = neighbours(g, p);
      const T gzm = g.nz > 1 ? gloc(phi[n.zm]) : (T)0, gzp = g.nz > 1 ? gloc(phi[n.zp]) : (T)0;
      const T lu = surf_lap(g, mc, n, u, gloc(f), gloc(phi[n.xm]), gloc(phi[n.xp]), gloc(phi[n.ym]),
                            gloc(phi[n.yp]), gzm, gzp);
      r += (mc.lambda_line / mc.mu) * (mc.eps_u * lu - gloc(f) * dW(uu) / mc.eps_u) * gn;
    }
    r += -(mc.M_area / mc.mu) * dvol * gn;
    r += (mc.alpha / mc.mu) * (uu + mc.u0) * gn * (e * L - Wp / e);
    out_rest[p] = r;
    out_wm[p] = Wm;
  }
}

// Membrane-velocity flux component d of g u v at q: v = -d_t phi grad phi / (|grad phi|^2 + 1e-12).
template <typename T>
__device__ __forceinline__ void adv_flux(const Geo& g, const ModelC<T>& mc, const T* __restrict__ phin,
                                         const T* __restrict__ phio, const T* __restrict__ u, int q,
                                         T& Fx, T& Fy, T& Fz) {
  const Nb n = neighbours(g, q);
  const T px = (phin[n.xp] - phin[n.xm]) * mc.i2h[0];
  const T py = (phin[n.yp] - phin[n.ym]) * mc.i2h[1];
  const T pz = g.nz > 1 ? (phin[n.zp] - phin[n.zm]) * mc.i2h[2] : (T)0;
  const T n2 = px * px + py * py + pz * pz + (T)1e-12;
  const T fq = phin[q];
  const T dt = (fq - phio[q]) / mc.tau;
  const T s = -gloc(fq) * u[q] * dt / n2;
  Fx = s * px;
  Fy = s * py;
  Fz = s * pz;
}

// R2 of the coupled OK equation (Sec. 3.1) at a band point p of phin.
template <typename T>
__device__ __forceinline__ T r2_coupled_at(const Geo& g, const ModelC<T>& mc, const T* __restrict__ phin,
                                           const T* __restrict__ phio, const T* __restrict__ u,
                                           const T* __restrict__ w, T mass, int p) {
  const T f = phin[p];
  const Nb n = neighbours(g, p);
  const T gc = gloc(f);
  const T gxm = gloc(phin[n.xm]), gxp = gloc(phin[n.xp]), gym = gloc(phin[n.ym]), gyp = gloc(phin[n.yp]);
  const T gzm = g.nz > 1 ? gloc(phin[n.zm]) : (T)0, gzp = g.nz > 1 ? gloc(phin[n.zp]) : (T)0;
  const T uc = u[p];
  const T sl = surf_lap(g, mc, n, u, gc, gxm, gxp, gym, gyp, gzm, gzp);
  const T guc = gc * uc;
  T lapgu = (gxp * u[n.xp] - (T)2 * guc + gxm * u[n.xm]) * mc.ih2[0] +
            (gyp * u[n.yp] - (T)2 * guc + gym * u[n.ym]) * mc.ih2[1];
  if (g.nz > 1) lapgu += (gzp * u[n.zp] - (T)2 * guc + gzm * u[n.zm]) * mc.ih2[2];
  T ax, ay, az, bx, by, bz;
  adv_flux(g, mc, phin, phio, u, n.xp, ax, ay, az);
  adv_flux(g, mc, phin, phio, u, n.xm, bx, by, bz);
  T div = (ax - bx) * mc.i2h[0];
  adv_flux(g, mc, phin, phio, u, n.yp, ax, ay, az);
  adv_flux(g, mc, phin, phio, u, n.ym, bx, by, bz);
  div += (ay - by) * mc.i2h[1];
  if (g.nz > 1) {
    adv_flux(g, mc, phin, phio, u, n.zp, ax, ay, az);
    adv_flux(g, mc, phin, phio, u, n.zm, bx, by, bz);
    div += (az - bz) * mc.i2h[2];
  }
  return mc.eps_u * (sl - mc.B1 * lapgu) + mc.B2 * guc - gc * dW(uc) / mc.eps_u - mc.gamma * gc * w[p] -
         mc.M * gc * mass - div;
}

// R2 on the band of phin over the whole grid, 0 elsewhere (operator entry point).
template <typename T>
__global__ void k_r2_coupled(Geo g, ModelC<T> mc, const T* __restrict__ phin, const T* __restrict__ phio,
                             const T* __restrict__ u, const T* __restrict__ w, const double* __restrict__ scal,
                             double hvol, T* __restrict__ out) {
  const T mass = (T)(hvol * scal[S_MASS]);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < (int)g.n; p += gridDim.x * blockDim.x) {
    const T f = phin[p];
    out[p] = (mc.linear_only || !in_band(f, mc.band_hi)) ? (T)0 : r2_coupled_at(g, mc, phin, phio, u, w, mass, p);
  }
}

// R2 at the points of the band list of phin only (the step: the rest of `out` was cleared
// when phin was formed).  Consecutive threads take consecutive band points, so the stencil
// work has no idle lanes.
template <typename T>
__global__ void k_r2_coupled_band(Geo g, ModelC<T> mc, const int* __restrict__ idx, const int* __restrict__ count,
                                  const T* __restrict__ phin, const T* __restrict__ phio, const T* __restrict__ u,
                                  const T* __restrict__ w, const double* __restrict__ scal, double hvol,
                                  T* __restrict__ out, unsigned long long* work) {
  const T mass = (T)(hvol * scal[S_MASS]);
  const int M = *count;
  if (work && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(work, (unsigned long long)M);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int p = idx[i];
    out[p] = mc.linear_only ? (T)0 : r2_coupled_at(g, mc, phin, phio, u, w, mass, p);
  }
}

// R2 of the fixed-membrane model: the Sec. 3 split of Eq. (2.1) with the operands of
// Eq. (2.16) (nonlocal operand g f(u), mass operand g (f(u) - ubar)); band from `mask`.
template <typename T>
__global__ void k_r2_fixed(Geo g, ModelC<T> mc, const T* __restrict__ G, const unsigned char* __restrict__ mask,
                           const T* __restrict__ u, const T* __restrict__ w, const double* __restrict__ scal,
                           double hvol, T* __restrict__ out) {
  const T mass = (T)(hvol * scal[S_MASS]);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < (int)g.n; p += gridDim.x * blockDim.x) {
    if (mc.linear_only || !mask[p]) {
      out[p] = 0;
      continue;
    }
    const Nb n = neighbours(g, p);
    const T gc = G[p];
    const T gxm = G[n.xm], gxp = G[n.xp], gym = G[n.ym], gyp = G[n.yp];
    const T gzm = g.nz > 1 ? G[n.zm] : (T)0, gzp = g.nz > 1 ? G[n.zp] : (T)0;
    const T uc = u[p];
    const T sl = surf_lap(g, mc, n, u, gc, gxm, gxp, gym, gyp, gzm, gzp);
    const T guc = gc * uc;
    T lapgu = (gxp * u[n.xp] - (T)2 * guc + gxm * u[n.xm]) * mc.ih2[0] +
              (gyp * u[n.yp] - (T)2 * guc + gym * u[n.ym]) * mc.ih2[1];
    if (g.nz > 1) lapgu += (gzp * u[n.zp] - (T)2 * guc + gzm * u[n.zm]) * mc.ih2[2];
    const T fp = dfind(uc);
    out[p] = mc.eps_u * (sl - mc.B1 * lapgu) + mc.B2 * guc - gc * dW(uc) / mc.eps_u - mc.gamma * gc * fp * w[p] -
             mc.M * gc * fp * mass;
  }
}

static __global__ void k_zero_off_band(long long n, const unsigned char* __restrict__ mask, void* x, int elem) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    if (!mask[p]) {
      if (elem == 8) reinterpret_cast<double*>(x)[p] = 0.0;
      else reinterpret_cast<float*>(x)[p] = 0.0f;
    }
}

template <typename T>
__global__ void k_axpy(long long n, const T* __restrict__ a, T c, const T* __restrict__ b, T* __restrict__ out) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    out[p] = a[p] + c * b[p];
}

// A0 = <phi^0, 1>_h when the caller left it unset.
static __global__ void k_set_a0(double* scal, double hvol) { scal[S_A0] = hvol * scal[S_VOL]; }

template <typename T> __global__ void k_gloc(long long n, const T* __restrict__ phi, T* __restrict__ G) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    G[p] = gloc(phi[p]);
}

// ---- FP64 reductions ---------------------------------------------------------------------
// Per-thread compensated sum in the storage precision: hi collects the rounded partial sums,
// lo the exact rounding error of each addition (Knuth's two-sum) plus any small parts the
// caller adds.  In FP32 it carries about twice the working precision, so the FP64 sums of
// the few per-thread partials match an FP64 accumulation while the per-element work stays
// on the FP32 pipes (FP64 arithmetic is a small fraction of the FP32 rate on this part).
template <typename T> struct CompSum {
  T hi = 0, lo = 0;
  __device__ __forceinline__ void add(T x) {
    const T s = hi + x;
    const T bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ubar = hi + lo in the storage precision (lo = 0 in FP64).
template <typename T> struct Ubar {
  T hi, lo;
};
template <typename T> __host__ __device__ inline Ubar<T> split_ubar(double ubar) {
  const T hi = (T)ubar;
  return Ubar<T>{hi, (T)(ubar - (double)hi)};
}

// One term G (x - ubar) of the mass sum.  FP32 forms it to about twice FP32 precision: ubar
// split into hi + lo, d = x - ubar as d_hi + d_lo (two-sum with the high part, then the low
// part), g d = rounded product + its rounding error (an FMA) + g d_lo.
__device__ __forceinline__ void add_mass(CompSum<float>& cs, float x, float g, Ubar<float> ub) {
  const float dh = x - ub.hi;
  const float bp = dh - x;
  const float dl = ((x - (dh - bp)) + (-ub.hi - bp)) - ub.lo;
  const float pr = g * dh;
  const float pe = fmaf(g, dh, -pr);
  cs.add(pr);
  cs.lo += fmaf(g, dl, pe);
}
__device__ __forceinline__ void add_mass(CompSum<double>& cs, double x, double g, Ubar<double> ub) {
  cs.add(g * ((x - ub.hi) - ub.lo));
}

// mode 0: sum a ; 1: sum G (u - ubar) ; 2: sum G (f(u) - ubar).  FP64 storage sums in FP64;
// FP32 storage forms each term to about twice FP32 precision (ubar split into hi + lo, the
// product's rounding error from an FMA) and sums with CompSum.
template <typename T>
__global__ void k_reduce(long long n, int mode, const T* __restrict__ a, const T* __restrict__ G, double ubar,
                         double* dst) {
  if constexpr (sizeof(T) == 8) {
    double s = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
      if (mode == 0) s += (double)a[p];
      else if (mode == 1) s += (double)G[p] * ((double)a[p] - ubar);
      else s += (double)G[p] * ((double)find(a[p]) - ubar);
    }
    block_add(s, dst);
    return;
  }
  const Ubar<float> ub = split_ubar<float>(ubar);
  CompSum<float> cs;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    if (mode == 0) {
      cs.add((float)a[p]);
      continue;
    }
    add_mass(cs, mode == 1 ? (float)a[p] : (float)find(a[p]), (float)G[p], ub);
  }
  block_add(cs.value(), dst);
}

// ---- inverse-transform epilogues that also form a field sum ------------------------------
// The volume <phi, 1> and the mass sum G (u - ubar) of Sec. 3.3 (k_reduce modes 0 and 1)
// accumulate while pass A stores the field: a compensated sum over each row pair a thread
// stores (Part), folded into FP64 per-thread sums (Acc), one block sum per CTA added
// atomically at the end; the field is not read back.  The caller zeroes the targets.
template <typename T> struct Sums2 {
  CompSum<T> s0, s1;
};
struct Acc2 {
  double s0 = 0.0, s1 = 0.0;
};

template <typename T> struct EpiStoreVol {
  static constexpr bool kPrefetch = false, kSums = true;
  using Acc = Acc2;
  using Part = Sums2<T>;
  __device__ void prefetch(long long) const {}
  T* out;
  double* vol;
  __device__ void operator()(long long i, T v, Part& a) const {
    out[i] = v;
    a.s0.add(v);
  }
  __device__ void fold(Part& p, Acc& a) const { a.s0 += p.s0.value(); }
  __device__ void finish(Acc& a) const { block_add(a.s0, vol); }
};

// EpiPhiG plus the volume of phi^{n+1}.
template <typename T> struct EpiPhiGVol {
  static constexpr bool kPrefetch = false, kSums = true;
  using Acc = Acc2;
  using Part = Sums2<T>;
  __device__ void prefetch(long long) const {}
  T* phi;
  T* G;
  T* zero;
  double* vol;
  __device__ void operator()(long long i, T v, Part& a) const {
    phi[i] = v;
    G[i] = gloc(v);
    if (zero) zero[i] = 0;
    a.s0.add(v);
  }
  __device__ void fold(Part& p, Acc& a) const { a.s0 += p.s0.value(); }
  __device__ void finish(Acc& a) const { block_add(a.s0, vol); }
};

// EpiRecover plus the mass sum of (G, u~).
template <typename T> struct EpiRecoverMass {
  static constexpr bool kPrefetch = true, kSums = true;
  using Acc = Acc2;
  using Part = Sums2<T>;
  __device__ void prefetch(long long i) const {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(G + i));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(base + i));
  }
  T* out;
  const T* G;
  const T* base;
  T delta;
  Ubar<T> ub;
  double* mass;
  __device__ void operator()(long long i, T v, Part& a) const {
    const T gg = G[i];
    const T b = base[i];
    const T o = gg > delta ? b + div_inc(v, gg) : gg * b + v;
    out[i] = o;
    add_mass(a.s0, o, gg, ub);
  }
  __device__ void fold(Part& p, Acc& a) const { a.s0 += p.s0.value(); }
  __device__ void finish(Acc& a) const { block_add(a.s0, mass); }
};

// ---- double-float transforms of the membrane state (FP32-mixed form) ----------------------
// Pass-A prologue of the double-float forward transform of an FP32 field.
struct ProWiden {
  const float* a;
  __device__ dfloat operator()(long long i) const { return dfloat(a[i]); }
};

// phi^{n+1} from the inverse transform of the phi-stage increment (FP32-mixed form): the
// real-space phi is carried as hi + lo (hi the FP32 field the other kernels read, lo its
// FP32 remainder), phi^{n+1} = (phi^n_hi + phi^n_lo) + d in double-float; G = 18 (phi (phi -
// 1))^2 is formed from the double-float value with phi - 1 as (hi - 1) + lo (hi - 1 is exact
// for hi in [0.5, 2]), so 1 - phi near the inner edge of the membrane and phi near the outer
// edge both keep their relative accuracy in G.  Also clears the R2 field and forms the volume.
struct EpiPhiIncVol {
  static constexpr bool kPrefetch = true, kSums = true;
  using Acc = Acc2;
  using Part = Sums2<float>;
  __device__ void prefetch(long long i) const {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(cur + i));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(lo + i));
  }
  const float* cur;   // phi^n (high part)
  float* lo;          // low part, phi^n on entry, phi^{n+1} on exit (in place)
  float* nxt;         // phi^{n+1} (high part)
  float* G;
  float* zero;
  double* vol;
  __device__ void operator()(long long i, float d, Part& a) const {
    const dfloat p = add_f(dfloat(cur[i], lo[i]), d);
    const float m1 = __fadd_rn(__fsub_rn(p.hi, 1.0f), p.lo);
    const float q = p.hi * m1;
    nxt[i] = p.hi;
    lo[i] = p.lo;
    G[i] = 18.0f * q * q;
    if (zero) zero[i] = 0.0f;
    a.s0.add(p.hi);
  }
  __device__ void fold(Part& p, Acc& a) const { a.s0 += p.s0.value(); }
  __device__ void finish(Acc& a) const { block_add(a.s0, vol); }
};

// Energy terms of Eq. (2.16) except the nonlocal one, plus the bound statistics and <phi,1>.
template <typename T>
__global__ void k_energy_terms(Geo g, ModelC<T> mc, const T* __restrict__ G, const T* __restrict__ U,
                               const T* __restrict__ phi, double* scal) {
  double sg = 0, sw = 0, sm = 0, sv = 0;
  double mb = 0, mn = 1e300, mx = -1e300;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < (int)g.n; p += gridDim.x * blockDim.x) {
    const Nb n = neighbours(g, p);
    const double gc = G[p], uc = U[p];
    const double dx = (double)U[n.xp] - uc, dy = (double)U[n.yp] - uc;
    sg += 0.5 * (gc + (double)G[n.xp]) * dx * dx * (double)mc.ih2[0] + 0.5 * (gc + (double)G[n.yp]) * dy * dy * (double)mc.ih2[1];
    if (g.nz > 1) {
      const double dz = (double)U[n.zp] - uc;
      sg += 0.5 * (gc + (double)G[n.zp]) * dz * dz * (double)mc.ih2[2];
    }
    sw += gc * (double)Wpot(U[p]);
    sm += gc * ((double)find(U[p]) - (double)mc.ubar);
    sv += (double)phi[p];
    if (gc > (double)mc.delta) {
      mb = fmax(mb, fabs(2.0 * uc - 1.0));
      mn = fmin(mn, uc);
      mx = fmax(mx, uc);
    }
  }
  block_add(sg, scal + S_GRAD);
  block_add(sw, scal + S_WELL);
  block_add(sm, scal + S_MASSF);
  block_add(sv, scal + S_VOLE);
  atomic_max_nonneg(scal + S_MAXB, mb);
  atomic_min_d(scal + S_UMIN, mn);
  atomic_max_d(scal + S_UMAX, mx);
}

template <typename T>
__global__ void k_check_finite(long long n, const T* __restrict__ a, int* flag) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    if (!isfinite(a[p])) {
      atomicOr(flag, 1);
      return;
    }
}

// ---- narrow-band compaction: ballot + scan into an ascending index list ----------------
constexpr int kCompactBlock = 1024;

template <typename T>
__global__ void k_band_count(long long n, const T* __restrict__ phi, T hi, unsigned char* __restrict__ mask,
                             int* __restrict__ bcount) {
  const long long p = blockIdx.x * (long long)kCompactBlock + threadIdx.x;
  const bool b = (p < n) && in_band(phi[p], hi);
  if (p < n) mask[p] = b ? 1 : 0;
  const unsigned bal = __ballot_sync(0xffffffffu, b);
  __shared__ int wc[32];
  if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = __popc(bal);
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = wc[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) bcount[blockIdx.x] = v;
  }
}

// The grid's band, 4 points per thread (one 16-byte load of phi per thread in FP32, one
// 4-byte mask store): a block covers kCompactWide consecutive points.  Needs n % 4 == 0 and
// a 16-byte aligned phi; k_band_scatter4 uses the same blocking.
constexpr int kCompactWide = 4 * kCompactBlock;

__device__ __forceinline__ void load4(const float* p, float (&f)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double (&f)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y;
}

template <typename T>
__global__ void k_band_count4(long long n, const T* __restrict__ phi, T hi, unsigned char* __restrict__ mask,
                              int* __restrict__ bcount) {
  const long long p0 = blockIdx.x * (long long)kCompactWide + 4LL * threadIdx.x;
  int c = 0;
  if (p0 < n) {
    T f[4];
    load4(phi + p0, f);
    uchar4 m;
    m.x = in_band(f[0], hi) ? 1 : 0;
    m.y = in_band(f[1], hi) ? 1 : 0;
    m.z = in_band(f[2], hi) ? 1 : 0;
    m.w = in_band(f[3], hi) ? 1 : 0;
    *reinterpret_cast<uchar4*>(mask + p0) = m;
    c = m.x + m.y + m.z + m.w;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  __shared__ int wc[32];
  if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = (threadIdx.x < (blockDim.x >> 5)) ? wc[threadIdx.x] : 0;
    v = __reduce_add_sync(0xffffffffu, v);
    if (threadIdx.x == 0) bcount[blockIdx.x] = v;
  }
}

// Block counts of a uint8 mask, 4 points per thread (kCompactWide blocking; n % 4 == 0).
static __global__ void k_mask_count4(long long n, const unsigned char* __restrict__ mask, int* __restrict__ bcount) {
  const long long p0 = blockIdx.x * (long long)kCompactWide + 4LL * threadIdx.x;
  int c = 0;
  if (p0 < n) {
    const uchar4 m = *reinterpret_cast<const uchar4*>(mask + p0);
    c = m.x + m.y + m.z + m.w;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  __shared__ int wc[32];
  if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = (threadIdx.x < (blockDim.x >> 5)) ? wc[threadIdx.x] : 0;
    v = __reduce_add_sync(0xffffffffu, v);
    if (threadIdx.x == 0) bcount[blockIdx.x] = v;
  }
}

// Index list and inverse map from the mask, 4 points per thread, ascending (kCompactWide
// blocking, boff = exclusive block offsets).
static __global__ void k_band_scatter4(long long n, const unsigned char* __restrict__ mask,
                                       const int* __restrict__ boff, int* __restrict__ idx, int* __restrict__ bmap) {
  const long long p0 = blockIdx.x * (long long)kCompactWide + 4LL * threadIdx.x;
  uchar4 m = make_uchar4(0, 0, 0, 0);
  if (p0 < n) m = *reinterpret_cast<const uchar4*>(mask + p0);
  const int c = m.x + m.y + m.z + m.w;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  __shared__ int wc[32];
  if (lane == 31) wc[wid] = inc;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int v = (lane < (int)(blockDim.x >> 5)) ? wc[lane] : 0;
    int w = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    wc[lane] = w - v;
  }
  __syncthreads();
  int i = boff[blockIdx.x] + wc[wid] + inc - c;
  const unsigned char mm[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
  for (int e = 0; e < 4; ++e)
    if (mm[e]) {
      idx[i] = (int)(p0 + e);
      bmap[p0 + e] = i;
      ++i;
    }
}

// Block counts of a uint8 mask (same blocking as k_band_count).
static __global__ void k_mask_count(long long n, const unsigned char* __restrict__ mask, int* __restrict__ bcount) {
  const long long p = blockIdx.x * (long long)kCompactBlock + threadIdx.x;
  const bool b = (p < n) && mask[p];
  const unsigned bal = __ballot_sync(0xffffffffu, b);
  __shared__ int wc[32];
  if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = __popc(bal);
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = wc[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) bcount[blockIdx.x] = v;
  }
}

// Exclusive scan of nb block counts in place (single block); total -> *count.
static __global__ void k_band_scan(int nb, int* __restrict__ bcount, int* __restrict__ count) {
  __shared__ int part[1024];
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per, hi = min(nb, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += bcount[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    const int v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;
  for (int i = lo; i < hi; ++i) {
    const int c = bcount[i];
    bcount[i] = run;
    run += c;
  }
  if (threadIdx.x == blockDim.x - 1) *count = part[threadIdx.x];
}

static __global__ void k_band_scatter(long long n, const unsigned char* __restrict__ mask, const int* __restrict__ boff,
                               int* __restrict__ idx, int* __restrict__ bmap) {
  const long long p = blockIdx.x * (long long)kCompactBlock + threadIdx.x;
  const bool b = (p < n) && mask[p];
  const unsigned bal = __ballot_sync(0xffffffffu, b);
  __shared__ int wc[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wc[wid] = __popc(bal);
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = wc[lane];
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    wc[lane] = inc - v;
  }
  __syncthreads();
  if (b) {
    const int i = boff[blockIdx.x] + wc[wid] + __popc(bal & ((1u << lane) - 1u));
    idx[i] = (int)p;
    bmap[p] = i;
  }
}

// ---- band CG for (-Delta_{S,h}) w = f - mean on the band ---------------------------------
// The band operator in compact form: for band node i (grid point p = idx[i]) and each of its
// 2d faces, c = (G_p + G_q)/(2 h^2) when the neighbour q is also a band node, else 0 (zero
// flux across the band edge); (A v)_i = sum_faces c (v_i - v_q).  Vectors are compact
// (length M, band order), so every CG phase streams contiguous arrays.
template <typename T> struct CGVec {
  T *x, *r, *u, *p, *q;   // compact vectors; q holds s = A p
  T* r1;                  // second residual buffer (the multigrid iterations alternate r, r1)
  T* idg;                 // inverse diagonal
  T* c;                   // face coefficients, c[d * cap + i], d = x+, x-, y+, y-, z+, z-
  __half* c16;            // the same in FP16 for the multigrid sweeps (FP32 storage only, else null)
  int* nb;                // compact index of the face neighbour (i itself when absent)
  int cap;
};

template <typename T>
__global__ void k_cg_setup(Geo g, ModelC<T> mc, const int* __restrict__ idx, const int* __restrict__ count,
                           const unsigned char* __restrict__ mask, const int* __restrict__ bmap,
                           const T* __restrict__ G, CGVec<T> v) {
  const int M = *count;
  const int nd = g.nz > 1 ? 6 : 4;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int p = idx[i];
    const Nb n = neighbours(g, p);
    const int q[6] = {n.xp, n.xm, n.yp, n.ym, n.zp, n.zm};
    const T gc = G[p];
    T d = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      T c = 0;
      int j = i;
      if (f < nd && mask[q[f]]) {
        c = (T)0.5 * (gc + G[q[f]]) * mc.ih2[f >> 1];
        j = bmap[q[f]];
      }
      v.c[f * v.cap + i] = c;
      if (v.c16) v.c16[f * v.cap + i] = __float2half_rn((float)c);
      v.nb[f * v.cap + i] = j;
      d += c;
    }
    v.idg[i] = d > (T)0 ? (T)1 / d : (T)1;
  }
}

// Zero the solution on nodes of the previous band that left the band.
static __global__ void k_zero_left(const int* __restrict__ old_idx, const int* __restrict__ old_count,
                            const unsigned char* __restrict__ mask, void* x, int elem) {
  const int M = *old_count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int p = old_idx[i];
    if (!mask[p]) {
      if (elem == 8) reinterpret_cast<double*>(x)[p] = 0.0;
      else reinterpret_cast<float*>(x)[p] = 0.0f;
    }
  }
}

// ---- connected components of the band (per-component mean removal of the band solve) ----
// The band operator is singular on every connected band component (6-neighbour, periodic),
// so the right-hand side and the solution are projected to zero mean per component (the
// whole-domain mean removal of Sec. 2.1 applied to each component).  Components come from a
// lock-free union-find over the band's neighbour lists: every link points from a larger node
// index to a smaller one, so each chase follows strictly decreasing indices and ends, and a
// failed link means another thread made progress (each loop is bounded by the node count).
constexpr int kCompCap = 4096;   // components the band solve supports (more: status 8)

__device__ __forceinline__ int cc_root(int* __restrict__ parent, int v) {
  int cur = __ldcg(parent + v);
  if (cur == v) return v;
  int prev = v;
  for (;;) {
    const int next = __ldcg(parent + cur);
    if (next >= cur) break;                // cur is a root (parent[cur] == cur)
    parent[prev] = next;                   // path halving; the value only ever decreases
    prev = cur;
    cur = next;
  }
  return cur;
}

// Each node starts as a child of its smallest band neighbour (or of itself), which leaves a
// forest with one tree per local minimum of the index over the band; linking then only has to
// merge those trees.
template <typename T>
__global__ void k_cc_init(const int* __restrict__ count, CGVec<T> v, int* __restrict__ parent, const int* fallback) {
  if (!*fallback) return;
  const int M = *count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    int m = i;
#pragma unroll
    for (int f = 0; f < 6; ++f) m = min(m, v.nb[f * v.cap + i]);
    parent[i] = m;
  }
}

template <typename T>
__global__ void k_cc_link(const int* __restrict__ count, CGVec<T> v, int* __restrict__ parent, int* status,
                          const int* fallback) {
  if (!*fallback) return;
  const int M = *count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int f = 0; f < 6; f += 2) {       // the + faces: every band edge is seen from one end
      const int j = v.nb[f * v.cap + i];
      if (j == i) continue;
      int a = cc_root(parent, i), b = cc_root(parent, j);
      for (int tries = 0; a != b; ++tries) {
        if (tries > M) {                   // cannot happen; guards the loop bound
          atomicCAS(status, 0, 8);
          return;
        }
        const int hi = a > b ? a : b, lo = a > b ? b : a;
        const int old = atomicCAS(parent + hi, hi, lo);
        if (old == hi) break;
        a = cc_root(parent, old);
        b = lo;
      }
    }
  }
}

// Full compression and a compact id per root (arbitrary order).
static __global__ void k_cc_roots(const int* __restrict__ count, int* __restrict__ parent, int* __restrict__ cid,
                                  int* __restrict__ ncomp, const int* fallback) {
  if (!*fallback) return;
  const int M = *count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int r = cc_root(parent, i);
    parent[i] = r;
    if (r == i) cid[i] = atomicAdd(ncomp, 1);
  }
}

// Per-component sums of one pass over the band: components below kCompShared accumulate in
// shared memory (one global atomic per block and component), others per warp group (lanes
// holding the same component combine their values, one atomic per group).  Every thread of
// the block calls begin() and end(); add() may be called under divergence.
constexpr int kCompShared = 64;
struct CompAcc {
  double* sh;    // kCompShared doubles of shared memory
  double* dst;   // global accumulators, one per component
  int C;
  __device__ void begin() {
    for (int k = threadIdx.x; k < kCompShared; k += blockDim.x) sh[k] = 0.0;
    __syncthreads();
  }
  __device__ void add(int c, double v) {
    if (c < kCompShared) {
      atomicAdd(sh + c, v);
      return;
    }
    const unsigned act = __activemask();
    const unsigned grp = __match_any_sync(act, c);
    double s = 0.0;
    for (unsigned m = grp; m; m &= m - 1) s += __shfl_sync(grp, v, __ffs(m) - 1);
    if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(dst + c, s);
  }
  __device__ void end() {
    __syncthreads();
    const int n = C < kCompShared ? C : kCompShared;
    for (int k = threadIdx.x; k < n; k += blockDim.x)
      if (sh[k] != 0.0) atomicAdd(dst + k, sh[k]);
    __syncthreads();
  }
};

// Node components and component sizes.  A band of one component needs neither: the solve
// then removes the plain mean, and only the size is written.
static __global__ void k_cc_label(const int* __restrict__ count, const int* __restrict__ parent,
                                  const int* __restrict__ cid, const int* __restrict__ ncomp, int* __restrict__ comp,
                                  double* __restrict__ csize, int* status, const int* fallback) {
  __shared__ double sh[kCompShared];
  if (!*fallback) return;
  const int M = *count;
  const int C = *ncomp;
  if (C > kCompCap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(status, 0, 8);
    return;
  }
  if (C <= 1) {
    if (blockIdx.x == 0 && threadIdx.x == 0) csize[0] = (double)M;
    return;
  }
  CompAcc acc{sh, csize, C};
  acc.begin();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int c = cid[parent[i]];
    comp[i] = c;
    acc.add(c, 1.0);
  }
  acc.end();
}

// Components from the multigrid hierarchy of the band solve.  A node of level l+1 is a 2x2x2
// cell of level-l nodes, and two level-(l+1) nodes are coupled exactly when a level-l coupling
// crosses between them.  If the children of every cell are connected inside the cell, the
// components of each level are the components of the next coarser one, so labelling the
// coarsest level (at most kCCCoarse nodes, one block) and following each band node's chain of
// parents gives the band's components.  A cell whose children split inside it, or a coarsest
// level that does not fit one block, sets the fallback flag and the union-find above runs.
constexpr int kCCCoarse = 1024;
constexpr int kCCMaxLev = 7;

struct CCLevel {
  const int* cnt;     // node count
  const int* nb;      // neighbour node of each face (the node itself where there is no coupling)
  const int* child;   // child[k * cap + I]: node of the finer level in sub-cell k, -1 if none
  const int* agg;     // parent node on the next coarser level
  int cap;
};
struct CCLevels {
  int nlev, is3d;
  CCLevel L[kCCMaxLev];
};

// Are the children of each cell connected inside it?  Sub-cell k = a + 2 b + 4 c (x, y, z bits);
// its in-cell neighbour across axis d is k ^ (1 << d), reached through face 2 d (+) when bit d of
// k is 0 and face 2 d + 1 (-) when it is 1.
static __global__ void k_cc_check(CCLevels lv, int* fallback) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  const int nax = lv.is3d ? 3 : 2;
  for (int l = 0; l + 1 < lv.nlev; ++l) {
    const CCLevel& F = lv.L[l];
    const CCLevel& Cl = lv.L[l + 1];
    const int Mc = *Cl.cnt;
    for (int I = tid; I < Mc; I += nth) {
      int ch[8];
      unsigned pres = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        ch[k] = Cl.child[k * Cl.cap + I];
        if (ch[k] >= 0) pres |= 1u << k;
      }
      if (__popc(pres) <= 1) continue;
      unsigned adj[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        adj[k] = 0;
        if (!((pres >> k) & 1)) continue;
        for (int d = 0; d < nax; ++d) {
          const int k2 = k ^ (1 << d);
          if (!((pres >> k2) & 1)) continue;
          const int f = 2 * d + ((k >> d) & 1);
          if (F.nb[f * F.cap + ch[k]] == ch[k2]) adj[k] |= 1u << k2;
        }
      }
      unsigned r = pres & (~pres + 1u);   // lowest present sub-cell
#pragma unroll
      for (int it = 0; it < 3; ++it) {    // the cube graph has diameter 3
        unsigned nr = r;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if ((r >> k) & 1) nr |= adj[k];
        r = nr;
      }
      if (r != pres) atomicExch(fallback, 1);
    }
  }
}

// Label the coarsest level in one block: min-label propagation with pointer jumping (bounded
// by the node count), compact ids of the roots, the component count.
static __global__ void __launch_bounds__(kCCCoarse) k_cc_coarsest(CCLevels lv, int* __restrict__ ccL,
                                                                  int* __restrict__ ncomp, int* fallback) {
  __shared__ int lab[kCCCoarse];
  __shared__ int cid[kCCCoarse];
  __shared__ int nroot;
  if (*(volatile int*)fallback) return;
  const CCLevel& L = lv.L[lv.nlev - 1];
  const int M = *L.cnt;
  if (M > kCCCoarse) {
    if (threadIdx.x == 0) atomicExch(fallback, 1);
    return;
  }
  const int i = threadIdx.x;
  if (i < M) lab[i] = i;
  if (i == 0) nroot = 0;
  __syncthreads();
  for (int it = 0; it <= M; ++it) {
    int m = i < M ? lab[i] : 0;
    if (i < M) {
      for (int f = 0; f < 6; ++f) {
        const int j = L.nb[f * L.cap + i];
        if (j != i) m = min(m, lab[j]);
      }
      m = min(m, lab[m]);
    }
    __syncthreads();
    const bool ch = i < M && m < lab[i];
    if (ch) lab[i] = m;
    if (!__syncthreads_or(ch)) break;
  }
  if (i < M && lab[i] == i) cid[i] = atomicAdd(&nroot, 1);
  __syncthreads();
  if (i < M) ccL[i] = cid[lab[i]];
  if (i == 0) *ncomp = nroot;
}

// Each band node's component through its chain of parents; the component sizes.
static __global__ void k_cc_down(CCLevels lv, const int* __restrict__ ccL, const int* __restrict__ ncomp,
                                 int* __restrict__ comp, double* __restrict__ csize, const int* fallback) {
  __shared__ double sh[kCompShared];
  if (*fallback) return;
  const int M = *lv.L[0].cnt;
  const int C = *ncomp;
  if (C <= 1) {
    if (blockIdx.x == 0 && threadIdx.x == 0) csize[0] = (double)M;
    return;
  }
  CompAcc acc{sh, csize, C};
  acc.begin();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    int j = i;
    for (int l = 0; l + 1 < lv.nlev; ++l) j = lv.L[l].agg[j];
    const int c = ccL[j];
    comp[i] = c;
    acc.add(c, 1.0);
  }
  acc.end();
}

template <typename T>
__device__ __forceinline__ T band_apply(const CGVec<T>& v, const T* __restrict__ a, int i) {
  const T ai = __ldcg(a + i);
  T s = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) s += v.c[f * v.cap + i] * (ai - __ldcg(a + v.nb[f * v.cap + i]));
  return s;
}

// Right-hand sides f of the band solve.
template <typename T> struct RhsField {
  const T* f;
  __device__ double operator()(long long p) const { return (double)f[p]; }
};
template <typename T> struct RhsGU {  // G (u - ubar): coupled nonlocal operand (Eq. (1.2))
  const T* G;
  const T* u;
  double ubar;
  __device__ double operator()(long long p) const { return (double)G[p] * ((double)u[p] - ubar); }
};
template <typename T> struct RhsGF {  // G f(u): fixed-model operand (Eq. (2.16))
  const T* G;
  const T* u;
  __device__ double operator()(long long p) const { return (double)G[p] * (double)find(u[p]); }
};

struct CGCtl {
  double* acc;          // 16 FP64 accumulators (zeroed before launch)
  unsigned* bar;        // [0] monotonic arrival count
  int* status;          // plan status word
  int* iters;           // out: iterations
  double* resid;        // out: relative residual
  double rtol;
  int maxit;
  long long budget;     // clock cycles a barrier may wait
  unsigned long long* work;  // accumulates band nodes x CG iterations (measurement)
  const int* ncomp;     // connected band components (device)
  const int* comp;      // component of each band node
  const double* csize;  // nodes per component
  double* csum;         // 2 kCompCap FP64 accumulators (zeroed before launch): f, then x
};

// Inside the band CG kernel every vector that the kernel itself writes (x, r, u, p, q and
// the multigrid levels' b, e, o, t) is read with __ldcg: an L2 load, never the read-only
// path that a const __restrict__ pointer would allow, which is only valid for data that no
// thread writes during the launch.  The couplings, neighbour lists and level maps are built
// by earlier launches and are read normally.

// Grid-wide barrier for a cooperative launch on one monotonic arrival counter (zeroed
// before the launch): barrier number e completes when the counter reaches e * gridDim.x,
// and each block learns e from the value its own arrival returned, so nothing is reset
// between barriers.  The block's writes are published by the block barrier followed by an
// acquire-release add at GPU scope; blocks that arrive early poll with acquire loads, and
// the last one to arrive takes its acquire from the add itself (without it, its L1 could
// still hold lines that other blocks rewrote during the phase).  The spin has a
// clock budget: when it runs out the kernel records ETD_ETIMEOUT in the status word and
// every block returns at its next check.  Returns false once the status is non-zero.
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_sync(const CGCtl& c) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const unsigned nb = gridDim.x;
    const unsigned old = atom_add_acq_rel_gpu(c.bar, 1u);
    const unsigned target = (old / nb + 1u) * nb;
    if (old + 1u != target) {
      const long long t0 = clock64();
      while ((int)(ld_acquire_gpu(c.bar) - target) < 0) {
        if (clock64() - t0 > c.budget) {
          atomicCAS(c.status, 0, 6);
          break;
        }
        __nanosleep(32);
      }
    }
    ok = (*(volatile int*)c.status == 0);
  }
  __syncthreads();
  return ok;
}

// ---- aggregation multigrid preconditioner for the band CG ---------------------------------
// Level l lives on the grid coarsened 2x per axis l times (z only in 3D); its nodes are the
// cells that contain at least one node of level l-1 (an aggregate of up to 2x2x2 nodes).
// With piecewise-constant prolongation P the Galerkin operator P^T A P of a graph Laplacian
// is again a graph Laplacian whose coupling between two neighbouring aggregates is the sum
// of the fine couplings crossing between them, so every level keeps the 7-point compact
// form (c, nb, inverse diagonal).  The preconditioner is one symmetric V(nu,nu) cycle whose
// smoother is weighted Jacobi; with nu = 2 the two sweeps use the weight pair w1, w2 of the
// degree-2 Chebyshev polynomial in D^-1 A (the two sweeps commute, so the cycle stays
// symmetric), and the coarsest level takes an even number of sweeps with the same pair.
constexpr int kMGMax = 7;

template <typename T> struct MGL {
  const int* cnt;      // node count (device)
  const int* list;     // flat cell index of each node on this level's grid
  const T* c;          // couplings c[f * cap + i]
  const int* nb;       // neighbour node of each face (i itself when absent)
  const T* idg;        // inverse diagonal
  int cap;
  const int* agg;      // parent node on level l+1 (l < nlev-1)
  const int* child;    // child[k * cap + I]: node of level l-1 in sub-cell k, -1 if none (l >= 1)
  T* b;                // right-hand side (level 0: the CG residual r)
  T* e;                // pre-smoothed correction
  T* o;                // output correction (level 0: the preconditioned residual u)
  T* t;                // scratch: residual handed to the restriction, first post-sweep
};

template <typename T> struct MGP {
  int nlev;            // 1 = plain Jacobi
  int gl;              // levels 0..gl-1 are processed by the whole grid, the rest by block 0
  int csweeps;         // Jacobi sweeps on the coarsest level (even)
  int nu;              // pre- and post-smoothing sweeps (1 or 2)
  T w1, w2;            // Jacobi weights of the first and second sweep (one Chebyshev pair)
  T alpha;             // over-correction of the coarse-grid correction
  const __half* c16;   // level-0 couplings in FP16 for the sweeps (null: use L[0].c)
  MGL<T> L[kMGMax];
};

// Multigrid set-up steps, written for any grid-stride partition (t0, ns) so that the large
// levels run them as grid-wide kernels and the small ones all inside one block.

// Extents of one level's grid (any even sizes; level l halves level l-1 along every axis,
// z only in 3D).
struct Ext {
  int x, y, z;
};
// The cell of level l holding flat index p of level l-1.
__device__ __forceinline__ int mg_cell(int p, Ext f, int is3d, Ext c) {
  const int X = p % f.x, t = p / f.x, Y = t % f.y, Z = t / f.y;
  return ((is3d ? Z >> 1 : 0) * c.y + (Y >> 1)) * c.x + (X >> 1);
}

// mark the cells of level l (extents c) holding nodes of level l-1 (extents f)
__device__ __forceinline__ void mg_mark_body(const int* __restrict__ list, int M, Ext f, int is3d, Ext c,
                                             unsigned char* __restrict__ mark, int t0, int ns) {
#pragma unroll 4
  for (int i = t0; i < M; i += ns) mark[mg_cell(list[i], f, is3d, c)] = 1;
}

__device__ __forceinline__ void mg_parent_body(const int* __restrict__ list, int M, Ext f, int is3d, Ext c,
                                               const int* __restrict__ cmap, int* __restrict__ agg, int t0, int ns) {
#pragma unroll 4
  for (int i = t0; i < M; i += ns) agg[i] = cmap[mg_cell(list[i], f, is3d, c)];
}

// Galerkin couplings of level l from level l-1.
template <typename T>
__device__ __forceinline__ void mg_coarse_body(const int* __restrict__ clist, int M, Ext ec, int is3d,
                                               const unsigned char* __restrict__ fmark,
                                               const int* __restrict__ fmap, Ext ef,
                                               const T* __restrict__ fc, int fcap, const int* __restrict__ cmap,
                                               T* __restrict__ c, int* __restrict__ nb, T* __restrict__ idg,
                                               int* __restrict__ child, int cap, int t0, int ns) {
  for (int I = t0; I < M; I += ns) {
    const int C = clist[I];
    const int X = C % ec.x, tq = C / ec.x, Y = tq % ec.y, Z = tq / ec.y;
    T s[6] = {0, 0, 0, 0, 0, 0};
    // the 8 children's marks, then their indices, then their couplings: three rounds of
    // independent loads instead of a dependent chain per child
    int Fk[8], jk[8];
    unsigned char mk[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int a = k & 1, b = (k >> 1) & 1, cz = k >> 2;
      Fk[k] = ((2 * Z + cz) * ef.y + (2 * Y + b)) * ef.x + (2 * X + a);
      mk[k] = (is3d || cz == 0) ? fmark[Fk[k]] : (unsigned char)0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) jk[k] = mk[k] ? fmap[Fk[k]] : -1;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int a = k & 1, b = (k >> 1) & 1, cz = k >> 2;
      const int j = jk[k];
      child[k * cap + I] = j;
      if (j < 0) continue;
      s[a ? 0 : 1] += fc[(a ? 0 : 1) * fcap + j];
      s[b ? 2 : 3] += fc[(b ? 2 : 3) * fcap + j];
      if (is3d) s[cz ? 4 : 5] += fc[(cz ? 4 : 5) * fcap + j];
    }
    const int xp = X + 1 == ec.x ? 0 : X + 1, xm = X == 0 ? ec.x - 1 : X - 1;
    const int yp = Y + 1 == ec.y ? 0 : Y + 1, ym = Y == 0 ? ec.y - 1 : Y - 1;
    const int zp = Z + 1 == ec.z ? 0 : Z + 1, zm = Z == 0 ? ec.z - 1 : Z - 1;
    const int ncell[6] = {(Z * ec.y + Y) * ec.x + xp, (Z * ec.y + Y) * ec.x + xm, (Z * ec.y + yp) * ec.x + X,
                          (Z * ec.y + ym) * ec.x + X, (zp * ec.y + Y) * ec.x + X, (zm * ec.y + Y) * ec.x + X};
    T d = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      c[f * cap + I] = s[f];
      nb[f * cap + I] = s[f] > (T)0 ? cmap[ncell[f]] : I;
      d += s[f];
    }
    idg[I] = d > (T)0 ? (T)1 / d : (T)1;
  }
}

static __global__ void k_mg_mark(const int* __restrict__ list, const int* __restrict__ cnt, Ext f, int is3d, Ext c,
                                 unsigned char* __restrict__ mark) {
  mg_mark_body(list, *cnt, f, is3d, c, mark, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

static __global__ void k_mg_parent(const int* __restrict__ list, const int* __restrict__ cnt, Ext f, int is3d, Ext c,
                                   const int* __restrict__ cmap, int* __restrict__ agg) {
  mg_parent_body(list, *cnt, f, is3d, c, cmap, agg, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <typename T>
__global__ void k_mg_coarse(const int* __restrict__ clist, const int* __restrict__ ccnt, Ext ec, int is3d,
                            const unsigned char* __restrict__ fmark, const int* __restrict__ fmap, Ext ef,
                            const T* __restrict__ fc, int fcap, const int* __restrict__ cmap, T* __restrict__ c,
                            int* __restrict__ nb, T* __restrict__ idg, int* __restrict__ child, int cap) {
  mg_coarse_body<T>(clist, *ccnt, ec, is3d, fmark, fmap, ef, fc, fcap, cmap, c, nb, idg, child, cap,
                    blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// One level's arrays for the single-block set-up of the small levels.
template <typename T> struct MGSetLevel {
  Ext e;
  int cap;
  int* cnt;
  int* list;
  int* map;
  unsigned char* mark;
  T* c;
  int* nb;
  T* idg;
  int* agg;
  int* child;
};

template <typename T> struct MGSetTail {
  int first, nlev, is3d;
  MGSetLevel<T> L[kMGMax];
};

// Levels first..nlev-1 built in order by one block of 1024 threads: mark, compact (one
// contiguous chunk of cells per thread, block-wide exclusive scan), parent map of the
// finer level, Galerkin couplings.  The finer level of `first` is complete on entry.
template <typename T> __global__ void __launch_bounds__(1024) k_mg_setup_tail(MGSetTail<T> a) {
  __shared__ int part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int l = a.first; l < a.nlev; ++l) {
    const MGSetLevel<T>& F = a.L[l - 1];
    const MGSetLevel<T>& L = a.L[l];
    for (int i = tid; i < L.cap; i += nt) L.mark[i] = 0;
    __syncthreads();
    const int MF = *F.cnt;
    mg_mark_body(F.list, MF, F.e, a.is3d, L.e, L.mark, tid, nt);
    __syncthreads();
    const int per = (L.cap + nt - 1) / nt;
    const int lo = min(L.cap, tid * per), hi = min(L.cap, lo + per);
    int own = 0;
#pragma unroll 4
    for (int i = lo; i < hi; ++i) own += L.mark[i];
    part[tid] = own;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
      const int v = tid >= off ? part[tid - off] : 0;
      __syncthreads();
      part[tid] += v;
      __syncthreads();
    }
    int pos = part[tid] - own;
    for (int i = lo; i < hi; ++i)
      if (L.mark[i]) {
        L.list[pos] = i;
        L.map[i] = pos;
        ++pos;
      }
    if (tid == nt - 1) *L.cnt = part[tid];
    __syncthreads();
    const int M = part[nt - 1];
    mg_parent_body(F.list, MF, F.e, a.is3d, L.e, L.map, F.agg, tid, nt);
    mg_coarse_body<T>(L.list, M, L.e, a.is3d, F.mark, F.map, F.e, F.c, F.cap, L.map, L.c, L.nb,
                      L.idg, L.child, L.cap, tid, nt);
    __syncthreads();
  }
}

template <typename T> __device__ __forceinline__ T mg_apply(const MGL<T>& L, const T* __restrict__ v, int i) {
  const T vi = __ldcg(v + i);
  T s = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) s += L.c[f * L.cap + i] * (vi - __ldcg(v + L.nb[f * L.cap + i]));
  return s;
}

// Barrier between consecutive V-cycle phases: a grid barrier when either phase runs on the
// whole grid, a block barrier inside block 0 when both run on block 0 alone.  The first
// call is free: the caller has already synchronised the grid.
struct PhaseSync {
  bool prev, first;
  __device__ bool step(bool cur, const CGCtl& c) {
    const bool g = prev || cur;
    prev = cur;
    if (first) {
      first = false;
      return true;
    }
    if (g) return grid_sync(c);
    if (blockIdx.x == 0) __syncthreads();
    return true;
  }
};

// A level-0 coupling for the multigrid sweeps: the FP16 copy where there is one (the
// preconditioner tolerates its rounding; the CG operator itself keeps the FP32 couplings).
template <typename T>
__device__ __forceinline__ T mg_coef(const T* __restrict__ c, const __half* __restrict__ h, int k) {
  return h ? (T)__half2float(h[k]) : c[k];
}

// The CG update x += a p, r_new = r_old - a q folded into the first smoothing sweep of the
// V-cycle that preconditions r_new (the sweep needs r_new at the neighbours, which it
// recomputes from r_old and q there, so the separate update pass and its barrier go away).
template <typename T> struct CGFuse {
  bool on;
  const T* rold;
  T* x;
  const T* p;
  const T* q;
  T a;
  double* rr;       // accumulates (r_new, r_new)
  double tol2;      // stop when (r_new, r_new) <= tol2
  double* zero;     // a CG accumulator every block has finished reading: zeroed on the way
};

// u = V(b), one symmetric V(nu,nu) cycle (nu = 1 or 2 weighted-Jacobi sweeps before and
// after the coarse-grid correction, which is scaled by alpha) for the level-0 right-hand
// side b.  On entry b is complete and visible (or, with the fused CG update, r_old, q, p and
// x are); on return every block has written its share of u (level-0 o) and added its part of
// (b,u) to *ru.  Residuals of the pre-sweeps are carried algebraically: e1 = w D^-1 b,
// r1 = b - A e1 (needs b at the neighbours), e2 = e1 + w D^-1 r1, r2 = r1 - w A D^-1 r1
// (needs r1 at the neighbours).  Returns -1 if a barrier failed, 1 if the fused update met
// the tolerance (the cycle is abandoned, *rr_out holds (r_new, r_new)), else 0.
template <typename T>
__device__ __forceinline__ int mg_vcycle(const MGP<T>& mg, const CGCtl& c, T* __restrict__ b0, const CGFuse<T>& F, double* ru,
                         double* rr_out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  PhaseSync ps{true, true};
  const T w1 = mg.w1, w2 = mg.w2, al = mg.alpha;
  // after the barrier that follows the fused sweep: every block sees (r_new, r_new)
  auto fused_check = [&]() -> bool {
    const double rr = *(volatile double*)F.rr;
    *rr_out = rr;
    if (blockIdx.x == 0 && threadIdx.x == 0) *F.zero = 0.0;
    return rr <= F.tol2;
  };
  for (int l = 0; l < mg.nlev - 1; ++l) {
    const MGL<T>& L = mg.L[l];
    const MGL<T>& Cl = mg.L[l + 1];
    bool grid = l < mg.gl;
    int t0 = grid ? tid : threadIdx.x, ns = grid ? nth : blockDim.x;
    if (!ps.step(grid, c)) return -1;
    if (grid || blockIdx.x == 0) {
      T* __restrict__ r1out = mg.nu == 2 ? L.o : L.t;
      const T* __restrict__ Lidg = L.idg;
      const T* __restrict__ Lc = L.c;
      const __half* __restrict__ Lh = l == 0 ? mg.c16 : nullptr;
      const int* __restrict__ Lnb = L.nb;
      T* __restrict__ Le = L.e;
      const int M = *L.cnt, cap = L.cap;
      if (l == 0 && F.on) {
        const T* __restrict__ Ro = F.rold;
        const T* __restrict__ Q = F.q;
        const T* __restrict__ P = F.p;
        T* __restrict__ X = F.x;
        const T a = F.a;
        T rr = 0;  // per-thread partial in the storage precision (a few nodes per thread)
        for (int i = t0; i < M; i += ns) {
          const T bi = __ldcg(Ro + i) - a * __ldcg(Q + i);
          X[i] = __ldcg(X + i) + a * __ldcg(P + i);
          b0[i] = bi;
          rr += bi * bi;
          const T ei = w1 * Lidg[i] * bi;
          T s = 0;
#pragma unroll
          for (int f = 0; f < 6; ++f) {
            const int j = Lnb[f * cap + i];
            // FP32 couplings here: this sweep is gather-bound and the half loads measured slower
            s += Lc[f * cap + i] * (ei - w1 * Lidg[j] * (__ldcg(Ro + j) - a * __ldcg(Q + j)));
          }
          Le[i] = ei;
          r1out[i] = bi - s;
        }
        block_add((double)rr, F.rr);
      } else {
        const T* __restrict__ Lb = l == 0 ? b0 : L.b;
#pragma unroll 2
        for (int i = t0; i < M; i += ns) {
          const T bi = __ldcg(Lb + i);
          const T ei = w1 * Lidg[i] * bi;
          T s = 0;
#pragma unroll
          for (int f = 0; f < 6; ++f) {
            const int j = Lnb[f * cap + i];
            s += mg_coef(Lc, Lh, f * cap + i) * (ei - w1 * Lidg[j] * __ldcg(Lb + j));
          }
          Le[i] = ei;
          r1out[i] = bi - s;
        }
      }
      if (mg.nu == 2) {  // the second sweep accumulates into the coarse right-hand side
        const int Mc = *Cl.cnt;
        for (int I = t0; I < Mc; I += ns) Cl.b[I] = 0;
      }
    }
    if (mg.nu == 2) {
      // second sweep e2 = e1 + w D^-1 r1, its residual r2 = r1 - w A D^-1 r1 added to the
      // parent aggregate's right-hand side (the restriction of piecewise-constant P)
      if (!ps.step(grid, c)) return -1;
      if (l == 0 && F.on && fused_check()) return 1;
      if (grid || blockIdx.x == 0) {
        const T* __restrict__ Lo = L.o;
        const T* __restrict__ Lidg = L.idg;
        const T* __restrict__ Lc = L.c;
        const __half* __restrict__ Lh = l == 0 ? mg.c16 : nullptr;
        const int* __restrict__ Lnb = L.nb;
        const int* __restrict__ Lagg = L.agg;
        T* __restrict__ Le = L.e;
        T* Cb = Cl.b;
        const int M = *L.cnt, cap = L.cap;
#pragma unroll 2
        for (int i = t0; i < M; i += ns) {
          const T oi = __ldcg(Lo + i);
          const T di = Lidg[i] * oi;
          T s = 0;
#pragma unroll
          for (int f = 0; f < 6; ++f) {
            const int j = Lnb[f * cap + i];
            s += mg_coef(Lc, Lh, f * cap + i) * (di - Lidg[j] * __ldcg(Lo + j));
          }
          Le[i] = __ldcg(Le + i) + w2 * di;
          atomicAdd(Cb + Lagg[i], oi - w2 * s);
        }
      }
      continue;
    }
    grid = (l + 1) < mg.gl;
    t0 = grid ? tid : threadIdx.x;
    ns = grid ? nth : blockDim.x;
    if (!ps.step(grid, c)) return -1;
    if (l == 0 && F.on && fused_check()) return 1;
    if (grid || blockIdx.x == 0) {
      const int M = *Cl.cnt;
      for (int I = t0; I < M; I += ns) {
        T s = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = Cl.child[q * Cl.cap + I];
          if (j >= 0) s += __ldcg(L.t + j);
        }
        Cl.b[I] = s;
      }
    }
  }
  {
    const MGL<T>& L = mg.L[mg.nlev - 1];
    const bool grid = (mg.nlev - 1) < mg.gl;
    const int t0 = grid ? tid : threadIdx.x, ns = grid ? nth : blockDim.x;
    if (!ps.step(grid, c)) return -1;
    if (grid || blockIdx.x == 0) {
      const int M = *L.cnt;
      for (int i = t0; i < M; i += ns) L.e[i] = w1 * L.idg[i] * __ldcg(L.b + i);
    }
    for (int s = 1; s < mg.csweeps; ++s) {
      if (!ps.step(grid, c)) return -1;
      const T* src = (s & 1) ? L.e : L.o;
      T* dst = (s & 1) ? L.o : L.e;
      if (grid || blockIdx.x == 0) {
        const int M = *L.cnt;
        for (int i = t0; i < M; i += ns) dst[i] = __ldcg(src + i) + ((s & 1) ? w2 : w1) * L.idg[i] * (__ldcg(L.b + i) - mg_apply(L, src, i));
      }
    }
  }
  for (int l = mg.nlev - 2; l >= 0; --l) {
    const MGL<T>& L = mg.L[l];
    const MGL<T>& Cl = mg.L[l + 1];
    const bool grid = l < mg.gl;
    const int t0 = grid ? tid : threadIdx.x, ns = grid ? nth : blockDim.x;
    if (!ps.step(grid, c)) return -1;
    T acc = 0;
    if (grid || blockIdx.x == 0) {
      T* __restrict__ out = mg.nu == 2 ? L.t : L.o;
      const T* __restrict__ Le = L.e;
      const T* __restrict__ Co = Cl.o;
      const T* __restrict__ Lb = l == 0 ? b0 : L.b;
      const T* __restrict__ Lidg = L.idg;
      const T* __restrict__ Lc = L.c;
      const __half* __restrict__ Lh = l == 0 ? mg.c16 : nullptr;
      const int* __restrict__ Lnb = L.nb;
      const int* __restrict__ Lagg = L.agg;
      const int M = *L.cnt, cap = L.cap;
#pragma unroll 2
      for (int i = t0; i < M; i += ns) {
        const T ei = __ldcg(Le + i) + al * __ldcg(Co + Lagg[i]);
        T s = 0;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          const int j = Lnb[f * cap + i];
          s += mg_coef(Lc, Lh, f * cap + i) * (ei - (__ldcg(Le + j) + al * __ldcg(Co + Lagg[j])));
        }
        const T bi = __ldcg(Lb + i);
        const T o1 = ei + (mg.nu == 2 ? w2 : w1) * Lidg[i] * (bi - s);
        out[i] = o1;
        if (l == 0 && mg.nu == 1) acc += bi * o1;
      }
    }
    if (mg.nu == 2) {
      if (!ps.step(grid, c)) return -1;
      if (grid || blockIdx.x == 0) {
        const T* __restrict__ Lt = L.t;
        const T* __restrict__ Lb = l == 0 ? b0 : L.b;
        const T* __restrict__ Lidg = L.idg;
        const T* __restrict__ Lc = L.c;
        const __half* __restrict__ Lh = l == 0 ? mg.c16 : nullptr;
        const int* __restrict__ Lnb = L.nb;
        T* __restrict__ Lo = L.o;
        const int M = *L.cnt, cap = L.cap;
#pragma unroll 2
        for (int i = t0; i < M; i += ns) {
          const T ti = __ldcg(Lt + i);
          T s = 0;
#pragma unroll
          for (int f = 0; f < 6; ++f) s += mg_coef(Lc, Lh, f * cap + i) * (ti - __ldcg(Lt + Lnb[f * cap + i]));
          const T bi = __ldcg(Lb + i);
          const T o2 = ti + w1 * Lidg[i] * (bi - s);
          Lo[i] = o2;
          if (l == 0) acc += bi * o2;
        }
      }
    }
    if (l == 0) block_add((double)acc, ru);
  }
  return 0;
}

enum { A_SUMF = 0, A_BB = 1, A_RU0 = 2, A_RR0 = 3, A_DU0 = 4, A_RU = 5, A_RR = 7, A_DU = 9, A_SUMX = 11 };

// u = M^{-1} b with M = Jacobi (one level) or one multigrid V-cycle; adds (b,u) to *ru.
template <typename T>
__device__ __forceinline__ bool precond(const CGVec<T>& v, const MGP<T>& mg, const CGCtl& c, int M, T* b,
                                        double* ru) {
  if (mg.nlev > 1) {
    CGFuse<T> off{};
    double rr;
    return mg_vcycle(mg, c, b, off, ru, &rr) == 0;
  }
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  double acc = 0;
  for (int i = tid; i < M; i += nth) {
    const T bi = __ldcg(b + i);
    const T u = bi * v.idg[i];
    v.u[i] = u;
    acc += (double)bi * (double)u;
  }
  block_add(acc, ru);
  return true;
}

// Preconditioned conjugate gradients, Chronopoulos-Gear arrangement (the recurrence
// s = A p replaces the second matrix product of textbook CG):
//   A: x += a p, r -= a s, rr = (r,r)                 | barrier
//   u = M^{-1} r, gamma = (r,u)                       | barrier
//   B: w = A u, p = u + b p, s = w + b s, delta=(w,u) | barrier
//   b = gamma/gamma_old, a = gamma/(delta - b gamma/a_old)
// With the multigrid preconditioner, A is folded into the first sweep of the V-cycle and
// the residual alternates between two buffers (the sweep reads the old one at the
// neighbours while it writes the new one).
// Initial guess of a band solve, x0 = a + cb b + cc c over the band (b, c may be null), from
// earlier solutions kept on the full grid; the solution is also written to hist (if set).
template <typename T> struct CGGuess {
  const T* a;
  const T* b;
  const T* c;
  T cb, cc;
  T* hist;
};

template <typename T, typename Rhs>
__global__ void __launch_bounds__(1024, 1) k_cg(const int* __restrict__ idx, const int* __restrict__ count,
                                                CGVec<T> v, T* __restrict__ wfull, Rhs rhs, CGCtl c, MGP<T> mg,
                                                CGGuess<T> gs) {
  const int M = *count;
  if (M == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      *c.iters = 0;
      *c.resid = 0.0;
    }
    return;
  }
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  // one band component: the plain mean; several: the mean of each (Sec. 2.1 per component)
  const int C = c.ncomp ? *c.ncomp : 1;
  __shared__ double csh[kCompShared];
  CompAcc cacc{csh, c.csum, C};
  if (C > 1) cacc.begin();
  double s = 0;
  for (int i = tid; i < M; i += nth) {
    const int p = idx[i];
    T x0 = gs.a[p];
    if (gs.b) x0 += gs.cb * gs.b[p];
    if (gs.c) x0 += gs.cc * gs.c[p];
    v.x[i] = x0;
    const double f = rhs(p);
    v.r1[i] = (T)f;             // f kept for the residual pass
    if (C > 1) cacc.add(c.comp[i], (double)(T)f);
    else s += f;
  }
  if (C > 1) cacc.end();
  else block_add(s, c.acc + A_SUMF);
  if (!grid_sync(c)) return;
  const double meanf = *(volatile double*)(c.acc + A_SUMF) / M;
  double bb = 0, rr = 0;
  for (int i = tid; i < M; i += nth) {
    double mf = meanf;
    if (C > 1) {
      const int ci = c.comp[i];
      mf = __ldcg(c.csum + ci) / c.csize[ci];
    }
    const double b = (double)__ldcg(v.r1 + i) - mf;
    const T r = (T)(b - (double)band_apply(v, v.x, i));
    v.r[i] = r;
    bb += b * b;
    rr += (double)r * (double)r;
  }
  block_add(bb, c.acc + A_BB);
  block_add(rr, c.acc + A_RR0);
  if (!grid_sync(c)) return;
  bb = *(volatile double*)(c.acc + A_BB);
  rr = *(volatile double*)(c.acc + A_RR0);
  const double tol2 = c.rtol * c.rtol * bb;
  bool conv = (bb == 0.0) || (rr <= tol2);
  double gamma = 0, delta = 0, alpha = 0;
  if (!conv) {
    if (!precond(v, mg, c, M, v.r, c.acc + A_RU0)) return;
    if (!grid_sync(c)) return;
    gamma = *(volatile double*)(c.acc + A_RU0);
    double du = 0;
    for (int i = tid; i < M; i += nth) {
      const T w = band_apply(v, v.u, i);
      const T u = __ldcg(v.u + i);
      v.p[i] = u;
      v.q[i] = w;
      du += (double)w * (double)u;
    }
    block_add(du, c.acc + A_DU0);
    if (!grid_sync(c)) return;
    delta = *(volatile double*)(c.acc + A_DU0);
    if (!(delta > 0.0)) conv = true;
    alpha = conv ? 0.0 : gamma / delta;
  }
  const bool fuse = mg.nlev > 1;
  int k = 0;
  while (!conv && k < c.maxit) {
    const int par = k & 1;
    const T a = (T)alpha;
    if (fuse) {
      CGFuse<T> F{true, par ? v.r1 : v.r, v.x, v.p, v.q, a, c.acc + A_RR + par, tol2, c.acc + A_DU + (par ^ 1)};
      const int st = mg_vcycle(mg, c, par ? v.r : v.r1, F, c.acc + A_RU + par, &rr);
      if (st < 0) return;
      ++k;
      if (st == 1) {
        conv = true;
        break;
      }
    } else {
      double rrn = 0;
      {
        T* __restrict__ X = v.x;
        T* __restrict__ Rr = v.r;
        const T* __restrict__ P = v.p;
        const T* __restrict__ Q = v.q;
#pragma unroll 4
        for (int i = tid; i < M; i += nth) {
          X[i] = __ldcg(X + i) + a * __ldcg(P + i);
          const T r = __ldcg(Rr + i) - a * __ldcg(Q + i);
          Rr[i] = r;
          rrn += (double)r * (double)r;
        }
      }
      block_add(rrn, c.acc + A_RR + par);
      if (!grid_sync(c)) return;
      if (blockIdx.x == 0 && threadIdx.x == 0) c.acc[A_DU + (par ^ 1)] = 0.0;
      rr = *(volatile double*)(c.acc + A_RR + par);
      ++k;
      if (rr <= tol2) {
        conv = true;
        break;
      }
      if (!precond(v, mg, c, M, v.r, c.acc + A_RU + par)) return;
    }
    if (!grid_sync(c)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) c.acc[A_RR + par] = 0.0;
    const double gnew = *(volatile double*)(c.acc + A_RU + par);
    const double beta = gnew / gamma;
    const T bt = (T)beta;
    T dun = 0;
    {
      const T* __restrict__ U = v.u;
      const T* __restrict__ Cc = v.c;
      const int* __restrict__ Nb = v.nb;
      T* __restrict__ P = v.p;
      T* __restrict__ Q = v.q;
      const int cap = v.cap;
#pragma unroll 2
      for (int i = tid; i < M; i += nth) {
        const T u = __ldcg(U + i);
        T w = 0;
#pragma unroll
        for (int f = 0; f < 6; ++f) w += Cc[f * cap + i] * (u - __ldcg(U + Nb[f * cap + i]));
        P[i] = u + bt * __ldcg(P + i);
        Q[i] = w + bt * __ldcg(Q + i);
        dun += w * u;
      }
    }
    block_add((double)dun, c.acc + A_DU + par);
    if (!grid_sync(c)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) c.acc[A_RU + par] = 0.0;
    delta = *(volatile double*)(c.acc + A_DU + par);
    const double den = delta - beta * gnew / alpha;
    if (!(den > 0.0)) break;
    alpha = gnew / den;
    gamma = gnew;
  }
  // zero-mean projection of the solution (per band component)
  if (!grid_sync(c)) return;
  double sx = 0;
  if (C > 1) {
    cacc.dst = c.csum + kCompCap;
    cacc.begin();
  }
  for (int i = tid; i < M; i += nth) {
    if (C > 1) cacc.add(c.comp[i], (double)__ldcg(v.x + i));
    else sx += (double)__ldcg(v.x + i);
  }
  if (C > 1) cacc.end();
  else block_add(sx, c.acc + A_SUMX);
  if (!grid_sync(c)) return;
  const T mx = (T)(*(volatile double*)(c.acc + A_SUMX) / M);
  for (int i = tid; i < M; i += nth) {
    const int p = idx[i];
    T mi = mx;
    if (C > 1) {
      const int ci = c.comp[i];
      mi = (T)(__ldcg(c.csum + kCompCap + ci) / c.csize[ci]);
    }
    const T w = __ldcg(v.x + i) - mi;
    wfull[p] = w;
    if (gs.hist) gs.hist[p] = w;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *c.iters = k;
    *c.resid = bb > 0 ? sqrt(rr / bb) : 0.0;
    if (!conv) atomicCAS(c.status, 0, 5);
    atomicAdd(c.work, (unsigned long long)k * (unsigned long long)M);
  }
}

// <w, f>: sum over the band (the nonlocal energy term).
template <typename T, typename Rhs>
__global__ void k_band_dot(const int* __restrict__ idx, const int* __restrict__ count, const T* __restrict__ w,
                           Rhs rhs, double* dst) {
  const int M = *count;
  double s = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int p = idx[i];
    s += (double)w[p] * rhs(p);
  }
  block_add(s, dst);
}

}  // namespace etd
