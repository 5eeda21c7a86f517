// kernels.cuh -- pointwise terms, finite-difference band terms, band compaction, the band
// conjugate-gradient solve and FP64 reductions of the ETD membrane step.
#pragma once
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

// Periodic neighbours of flat index p.
struct Nb {
  long long c, xm, xp, ym, yp, zm, zp;
};
__device__ __forceinline__ Nb neighbours(const Geo& g, long long p) {
  const int x = (int)(p % g.nx);
  const long long t = p / g.nx;
  const int y = (int)(t % g.ny);
  const int z = (int)(t / g.ny);
  const long long row = p - x;
  const long long pl = (long long)g.nx * g.ny;
  const long long plane = p - (long long)y * g.nx - x;
  Nb n;
  n.c = p;
  n.xm = row + (x == 0 ? g.nx - 1 : x - 1);
  n.xp = row + (x == g.nx - 1 ? 0 : x + 1);
  n.ym = plane + (long long)(y == 0 ? g.ny - 1 : y - 1) * g.nx + x;
  n.yp = plane + (long long)(y == g.ny - 1 ? 0 : y + 1) * g.nx + x;
  if (g.nz > 1) {
    n.zm = (long long)(z == 0 ? g.nz - 1 : z - 1) * pl + (p - (long long)z * pl);
    n.zp = (long long)(z == g.nz - 1 ? 0 : z + 1) * pl + (p - (long long)z * pl);
  } else {
    n.zm = n.zp = p;
  }
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
  T* out;
  __device__ void operator()(long long i, T v) const { out[i] = v; }
};
// U = GU/G where G > delta, GU elsewhere (Sec. 3.3, recovery after Algorithm 1).
template <typename T> struct EpiRecover {
  T* out;
  const T* G;
  T delta;
  __device__ void operator()(long long i, T v) const {
    const T gg = G[i];
    out[i] = gg > delta ? v / gg : v;
  }
};
// phi^{n+1} and G^{n+1} = 18 (phi^2 - phi)^2 (Algorithm 1).
template <typename T> struct EpiPhiG {
  T* phi;
  T* G;
  __device__ void operator()(long long i, T v) const {
    phi[i] = v;
    G[i] = gloc(v);
  }
};

// ---- pointwise / band kernels ----------------------------------------------------------

// Lu = Delta_{S,h} u with g = g(phi), on the band of phi (0 elsewhere).
template <typename T>
__global__ void k_surf_lap_band(Geo g, ModelC<T> mc, const T* __restrict__ phi, const T* __restrict__ u,
                                T* __restrict__ out) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n; p += (long long)gridDim.x * blockDim.x) {
    const T f = phi[p];
    if (!in_band(f, mc.band_hi)) {
      out[p] = 0;
      continue;
    }
    const Nb n = neighbours(g, p);
    const T gz_m = g.nz > 1 ? gloc(phi[n.zm]) : (T)0, gz_p = g.nz > 1 ? gloc(phi[n.zp]) : (T)0;
    out[p] = surf_lap(g, mc, n, u, gloc(f), gloc(phi[n.xm]), gloc(phi[n.xp]), gloc(phi[n.ym]), gloc(phi[n.yp]),
                      gz_m, gz_p);
  }
}

// R1 without its Laplacian term (Sec. 3.1), and W'(phi) - A1 phi whose spectrum receives
// kappa/(mu eps^2) lambda in pass B.  Delta phi and grad phi are spectral (pass-A outputs).
template <typename T>
__global__ void k_r1(Geo g, ModelC<T> mc, const T* __restrict__ phi, const T* __restrict__ lap,
                     const T* __restrict__ gx, const T* __restrict__ gy, const T* __restrict__ gz,
                     const T* __restrict__ u, const T* __restrict__ lu, const double* __restrict__ scal,
                     double hvol, T* __restrict__ out_rest, T* __restrict__ out_wm) {
  const T e = mc.eps_phi, e2 = e * e;
  const T dvol = (T)(hvol * scal[S_VOL] - scal[S_A0]);
  const T c_a = mc.kappa / (mc.mu * e2);
  const T c_b = mc.kappa / (mc.mu * e2 * e2);
  const T c_c = mc.lambda_surf / (mc.mu * e2);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n; p += (long long)gridDim.x * blockDim.x) {
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
    if (in_band(f, mc.band_hi))
      r += (mc.lambda_line / mc.mu) * (mc.eps_u * lu[p] - gloc(f) * dW(uu) / mc.eps_u) * gn;
    r += -(mc.M_area / mc.mu) * dvol * gn;
    r += (mc.alpha / mc.mu) * (uu + mc.u0) * gn * (e * L - Wp / e);
    out_rest[p] = r;
    out_wm[p] = Wm;
  }
}

// Membrane-velocity flux component d of g u v at q: v = -d_t phi grad phi / (|grad phi|^2 + 1e-12).
template <typename T>
__device__ __forceinline__ void adv_flux(const Geo& g, const ModelC<T>& mc, const T* __restrict__ phin,
                                         const T* __restrict__ phio, const T* __restrict__ u, long long q,
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

// R2 of the coupled OK equation (Sec. 3.1) on the band of phin, 0 elsewhere.
template <typename T>
__global__ void k_r2_coupled(Geo g, ModelC<T> mc, const T* __restrict__ phin, const T* __restrict__ phio,
                             const T* __restrict__ u, const T* __restrict__ w, const double* __restrict__ scal,
                             double hvol, T* __restrict__ out) {
  const T mass = (T)(hvol * scal[S_MASS]);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n; p += (long long)gridDim.x * blockDim.x) {
    const T f = phin[p];
    if (mc.linear_only || !in_band(f, mc.band_hi)) {
      out[p] = 0;
      continue;
    }
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
    out[p] = mc.eps_u * (sl - mc.B1 * lapgu) + mc.B2 * guc - gc * dW(uc) / mc.eps_u - mc.gamma * gc * w[p] -
             mc.M * gc * mass - div;
  }
}

// R2 of the fixed-membrane model: the Sec. 3 split of Eq. (2.1) with the operands of
// Eq. (2.16) (nonlocal operand g f(u), mass operand g (f(u) - ubar)); band from `mask`.
template <typename T>
__global__ void k_r2_fixed(Geo g, ModelC<T> mc, const T* __restrict__ G, const unsigned char* __restrict__ mask,
                           const T* __restrict__ u, const T* __restrict__ w, const double* __restrict__ scal,
                           double hvol, T* __restrict__ out) {
  const T mass = (T)(hvol * scal[S_MASS]);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n; p += (long long)gridDim.x * blockDim.x) {
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
// mode 0: sum a ; 1: sum G (u - ubar) ; 2: sum G (f(u) - ubar)
template <typename T>
__global__ void k_reduce(long long n, int mode, const T* __restrict__ a, const T* __restrict__ G, double ubar,
                         double* dst) {
  double s = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    if (mode == 0) s += (double)a[p];
    else if (mode == 1) s += (double)G[p] * ((double)a[p] - ubar);
    else s += (double)G[p] * ((double)find(a[p]) - ubar);
  }
  block_add(s, dst);
}

// Energy terms of Eq. (2.16) except the nonlocal one, plus the bound statistics and <phi,1>.
template <typename T>
__global__ void k_energy_terms(Geo g, ModelC<T> mc, const T* __restrict__ G, const T* __restrict__ U,
                               const T* __restrict__ phi, double* scal) {
  double sg = 0, sw = 0, sm = 0, sv = 0;
  double mb = 0, mn = 1e300, mx = -1e300;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n; p += (long long)gridDim.x * blockDim.x) {
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
                               int* __restrict__ idx) {
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
  if (b) idx[boff[blockIdx.x] + wc[wid] + __popc(bal & ((1u << lane) - 1u))] = (int)p;
}

// ---- band CG for (-Delta_{S,h}) w = f - mean on the band ---------------------------------
// Face coefficients c_d(p) = (G_p + G_{p+e_d})/2 when p and p+e_d are both band nodes, else 0
// (zero flux across the band edge).  Vectors live in full-grid layout, band entries only.
template <typename T> struct CGVec {
  T *x, *r, *p, *q, *cx, *cy, *cz, *idg;
};

template <typename T>
__global__ void k_cg_setup(Geo g, ModelC<T> mc, const int* __restrict__ idx, const int* __restrict__ count,
                           const unsigned char* __restrict__ mask, const T* __restrict__ G, CGVec<T> v) {
  const int M = *count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const long long p = idx[i];
    const Nb n = neighbours(g, p);
    const T gc = G[p];
    v.cx[p] = mask[n.xp] ? (T)0.5 * (gc + G[n.xp]) : (T)0;
    v.cy[p] = mask[n.yp] ? (T)0.5 * (gc + G[n.yp]) : (T)0;
    if (!mask[n.xm]) v.cx[n.xm] = 0;
    if (!mask[n.ym]) v.cy[n.ym] = 0;
    if (g.nz > 1) {
      v.cz[p] = mask[n.zp] ? (T)0.5 * (gc + G[n.zp]) : (T)0;
      if (!mask[n.zm]) v.cz[n.zm] = 0;
    }
  }
}

template <typename T>
__global__ void k_cg_diag(Geo g, ModelC<T> mc, const int* __restrict__ idx, const int* __restrict__ count,
                          CGVec<T> v) {
  const int M = *count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const long long p = idx[i];
    const Nb n = neighbours(g, p);
    T d = (v.cx[p] + v.cx[n.xm]) * mc.ih2[0] + (v.cy[p] + v.cy[n.ym]) * mc.ih2[1];
    if (g.nz > 1) d += (v.cz[p] + v.cz[n.zm]) * mc.ih2[2];
    v.idg[p] = d > (T)0 ? (T)1 / d : (T)1;
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

template <typename T>
__device__ __forceinline__ T neg_lap_apply(const Geo& g, const ModelC<T>& mc, const CGVec<T>& v, const T* __restrict__ a,
                                           long long p) {
  const Nb n = neighbours(g, p);
  const T ac = a[p];
  T s = (v.cx[p] * (a[n.xp] - ac) - v.cx[n.xm] * (ac - a[n.xm])) * mc.ih2[0] +
        (v.cy[p] * (a[n.yp] - ac) - v.cy[n.ym] * (ac - a[n.ym])) * mc.ih2[1];
  if (g.nz > 1) s += (v.cz[p] * (a[n.zp] - ac) - v.cz[n.zm] * (ac - a[n.zm])) * mc.ih2[2];
  return -s;
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
  unsigned* bar;        // [0] arrival count, [1] generation
  int* status;          // plan status word
  int* iters;           // out: iterations
  double* resid;        // out: relative residual
  double rtol;
  int maxit;
  long long budget;     // clock cycles a barrier may wait
  unsigned long long* work;  // accumulates band nodes x sweeps (measurement)
};

// Grid-wide barrier for a cooperative launch.  The spin has a clock budget: when it runs
// out the kernel records ETD_ETIMEOUT in the status word and every block returns at its
// next check.  Returns false once the status is non-zero.
__device__ __forceinline__ bool grid_sync(const CGCtl& c) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = c.bar + 1;
    const unsigned my = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(c.bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(c.bar, 0u);
      __threadfence();
      atomicAdd(c.bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == my) {
        if (clock64() - t0 > c.budget) {
          atomicCAS(c.status, 0, 6);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = (*(volatile int*)c.status == 0);
  }
  __syncthreads();
  return ok;
}

enum { A_SUMF = 0, A_BB = 1, A_RZ0 = 2, A_RR0 = 3, A_PQ = 4, A_RZ = 6, A_RR = 8, A_SUMX = 10 };

template <typename T, typename Rhs>
__global__ void __launch_bounds__(256) k_cg(Geo g, ModelC<T> mc, const int* __restrict__ idx,
                                            const int* __restrict__ count, CGVec<T> v, Rhs rhs, CGCtl c) {
  const int M = *count;
  if (M == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      *c.iters = 0;
      *c.resid = 0.0;
    }
    return;
  }
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  double s = 0;
  for (int i = tid; i < M; i += nth) s += rhs(idx[i]);
  block_add(s, c.acc + A_SUMF);
  if (!grid_sync(c)) return;
  const double meanf = *(volatile double*)(c.acc + A_SUMF) / M;
  double bb = 0, rz = 0, rr = 0;
  for (int i = tid; i < M; i += nth) {
    const long long p = idx[i];
    const double b = rhs(p) - meanf;
    const T r = (T)(b - (double)neg_lap_apply(g, mc, v, v.x, p));
    const T z = r * v.idg[p];
    v.r[p] = r;
    v.p[p] = z;
    bb += b * b;
    rz += (double)r * (double)z;
    rr += (double)r * (double)r;
  }
  block_add(bb, c.acc + A_BB);
  block_add(rz, c.acc + A_RZ0);
  block_add(rr, c.acc + A_RR0);
  if (!grid_sync(c)) return;
  bb = *(volatile double*)(c.acc + A_BB);
  rz = *(volatile double*)(c.acc + A_RZ0);
  rr = *(volatile double*)(c.acc + A_RR0);
  const double tol2 = c.rtol * c.rtol * bb;
  int k = 0;
  bool conv = (bb == 0.0) || (rr <= tol2);
  while (!conv && k < c.maxit) {
    const int par = k & 1;
    double pq = 0;
    for (int i = tid; i < M; i += nth) {
      const long long p = idx[i];
      const T q = neg_lap_apply(g, mc, v, v.p, p);
      v.q[p] = q;
      pq += (double)v.p[p] * (double)q;
    }
    block_add(pq, c.acc + A_PQ + par);
    if (!grid_sync(c)) return;
    pq = *(volatile double*)(c.acc + A_PQ + par);
    if (!(pq > 0.0)) break;
    const T alpha = (T)(rz / pq);
    double rzn = 0, rrn = 0;
    for (int i = tid; i < M; i += nth) {
      const long long p = idx[i];
      v.x[p] += alpha * v.p[p];
      const T r = v.r[p] - alpha * v.q[p];
      v.r[p] = r;
      const T z = r * v.idg[p];
      rzn += (double)r * (double)z;
      rrn += (double)r * (double)r;
    }
    block_add(rzn, c.acc + A_RZ + par);
    block_add(rrn, c.acc + A_RR + par);
    if (!grid_sync(c)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) c.acc[A_PQ + par] = 0.0;
    rzn = *(volatile double*)(c.acc + A_RZ + par);
    rrn = *(volatile double*)(c.acc + A_RR + par);
    ++k;
    rr = rrn;
    if (rrn <= tol2) {
      conv = true;
      break;
    }
    const T beta = (T)(rzn / rz);
    rz = rzn;
    for (int i = tid; i < M; i += nth) {
      const long long p = idx[i];
      v.p[p] = v.r[p] * v.idg[p] + beta * v.p[p];
    }
    if (!grid_sync(c)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c.acc[A_RZ + par] = 0.0;
      c.acc[A_RR + par] = 0.0;
    }
  }
  // zero-mean projection of the solution (single band component)
  if (!grid_sync(c)) return;
  double sx = 0;
  for (int i = tid; i < M; i += nth) sx += (double)v.x[idx[i]];
  block_add(sx, c.acc + A_SUMX);
  if (!grid_sync(c)) return;
  const T mx = (T)(*(volatile double*)(c.acc + A_SUMX) / M);
  for (int i = tid; i < M; i += nth) v.x[idx[i]] -= mx;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *c.iters = k;
    *c.resid = bb > 0 ? sqrt(rr / bb) : 0.0;
    atomicAdd(c.work, (unsigned long long)(k + 3) * (unsigned long long)M);
    if (!conv) atomicCAS(c.status, 0, 5);
  }
}

// <w, f>: sum over the band (the nonlocal energy term).
template <typename T, typename Rhs>
__global__ void k_band_dot(const int* __restrict__ idx, const int* __restrict__ count, const T* __restrict__ w,
                           Rhs rhs, double* dst) {
  const int M = *count;
  double s = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const long long p = idx[i];
    s += (double)w[p] * rhs(p);
  }
  block_add(s, dst);
}

}  // namespace etd
