// krylov.cuh -- the g^{1/2}-split fixed-membrane scheme of Sec. 2.2 on the narrow band:
//   d V/dt + L V = R_phi(U),  V = g^{1/2} U,
//   L = B I - eps_u G^{-1/2} Delta_{S,h} G^{-1/2},
//   R_phi(U) = g^{1/2} (B U - W'(U)/eps_u - gamma f'(U) w - M m f'(U)),
//   w = (-Delta_{S,h})^{-1}(g f(U)) (the band solve), m = <g (f(U) - ubar), 1>_h,
// advanced by ETD1 (Eq. (2.8)) or ETDRK2 (Eq. (2.9)-(2.10)).  L is symmetric but not
// diagonal in Fourier space, so its matrix functions act through the Krylov space of the
// Lanczos process (Hochbruck-Lubich): phi_j(tau L) b ~ |b| V_m phi_j(tau T_m) e_1 with T_m the
// Lanczos tridiagonal matrix.  Since phi_0(z) = 1 - z phi_1(z), the first stage is taken as
//   V~ = V + tau phi_1(tau L) (R(U) - L V)
// (one Krylov space instead of two), the ETDRK2 corrector as V~ + tau phi_2(tau L)(R(U~) - R(U)).
// The band is the band solve's (zero flux across its edge): L x at band node i reads the
// face couplings c_f(i) = (g_i + g_j)/(2 h^2) and neighbour lists of the band solve's set-up.
// U off the band is not part of the system and is never written.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>
#include "kernels.cuh"

namespace etd {

constexpr int kKrylovMax = 128;   // largest Krylov dimension of one phi_j(tau L) b
constexpr int kKrylovChunk = 8;   // Lanczos steps per launch (a convergence check after each)

template <typename T> struct KrylovOp {
  CGVec<T> v;        // couplings and neighbour lists of the band (band solve's set-up)
  const T* isg;      // g^{-1/2} per band node
  T B, eps_u;
};

// (L x)_i for a compact vector x that the calling launch writes (read through L2).
template <typename T>
__device__ __forceinline__ T krylov_apply(const KrylovOp<T>& op, const T* x, int i) {
  const T xi = __ldcg(x + i), si = op.isg[i];
  T s = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int j = op.v.nb[f * op.v.cap + i];
    s += op.v.c[f * op.v.cap + i] * (si * xi - op.isg[j] * __ldcg(x + j));
  }
  return op.B * xi + op.eps_u * si * s;
}

// Lanczos steps j0 .. j1-1 on the basis V_j = V + j * ld (V_{j0} given; for j0 > 0 also V_{j0-1}
// and beta[j0-1] from the previous launch):
//   alpha_j = (L V_j, V_j),  w = L V_j - alpha_j V_j - beta_{j-1} V_{j-1},
//   beta_j = |w|,  V_{j+1} = w / beta_j.
// acc holds two FP64 accumulators per step (zeroed before the first launch of a Krylov space).
// beta_j = 0 (an invariant subspace) ends the process.  Cooperative launch; every grid
// barrier is bounded (status 6 when it gives up, then every block returns).
template <typename T>
__global__ void __launch_bounds__(1024, 1) k_lanczos(const int* __restrict__ count, KrylovOp<T> op, T* V, int ld,
                                                      T* w, double* alpha, double* beta, double* acc, int j0, int j1,
                                                      CGCtl c) {
  const int M = *count;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  T bprev = j0 > 0 ? (T)beta[j0 - 1] : (T)0;
  if (j0 > 0 && !(bprev > (T)0)) return;
  for (int j = j0; j < j1; ++j) {
    if (j > j0 && !grid_sync(c)) return;   // V_j complete at every node
    const T* Vj = V + (size_t)j * ld;
    const T* Vp = j > 0 ? V + (size_t)(j - 1) * ld : nullptr;
    double a = 0;
    for (int i = tid; i < M; i += nth) {
      T x = krylov_apply(op, Vj, i);
      if (Vp) x -= bprev * __ldcg(Vp + i);
      w[i] = x;
      a += (double)x * (double)__ldcg(Vj + i);
    }
    block_add(a, acc + 2 * j);
    if (!grid_sync(c)) return;
    const double al = *(volatile double*)(acc + 2 * j);
    double nn = 0;
    for (int i = tid; i < M; i += nth) {
      const T x = w[i] - (T)al * __ldcg(Vj + i);
      w[i] = x;
      nn += (double)x * (double)x;
    }
    block_add(nn, acc + 2 * j + 1);
    if (!grid_sync(c)) return;
    const double bb = sqrt(*(volatile double*)(acc + 2 * j + 1));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      alpha[j] = al;
      beta[j] = bb;
    }
    if (!(bb > 0.0)) return;
    const T ib = (T)(1.0 / bb);
    T* Vn = V + (size_t)(j + 1) * ld;
    for (int i = tid; i < M; i += nth) Vn[i] = w[i] * ib;
    bprev = (T)bb;
  }
}

// |x|^2 of a compact vector, added to *dst (zeroed by the caller).
template <typename T>
__global__ void k_band_norm2(const int* __restrict__ count, const T* __restrict__ x, double* dst) {
  const int M = *count;
  double s = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x)
    s += (double)x[i] * (double)x[i];
  block_add(s, dst);
}

// y = x / |x| with |x|^2 in *nrm2 (compact).
template <typename T>
__global__ void k_band_normalise(const int* __restrict__ count, const T* __restrict__ x, const double* __restrict__ nrm2,
                                 T* __restrict__ y) {
  const int M = *count;
  const double s = 1.0 / sqrt(*nrm2);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) y[i] = (T)(s * (double)x[i]);
}

// g^{1/2} and g^{-1/2} at the band nodes (g > 0 there: the band excludes g near 0).
template <typename T>
__global__ void k_sec2_sqrtg(const int* __restrict__ idx, const int* __restrict__ count, const T* __restrict__ G,
                             T* __restrict__ sg, T* __restrict__ isg) {
  const int M = *count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const double g = (double)G[idx[i]];
    sg[i] = (T)sqrt(g);
    isg[i] = (T)(1.0 / sqrt(g));
  }
}

// R_phi(U)_i - B g^{1/2} U_i: the nonlinear part of the remainder at band node i (0 when the
// nonlinear terms are switched off).
template <typename T>
__device__ __forceinline__ T sec2_nl(const ModelC<T>& mc, T s, T u, T w, T mass) {
  if (mc.linear_only) return (T)0;
  const T fp = dfind(u);
  return -s * (dW(u) / mc.eps_u + mc.gamma * fp * w + mc.M * mass * fp);
}

// First stage: R0 = R_phi(U) and b = R0 - L (g^{1/2} U) at the band nodes.  With V = g^{1/2} U,
// (L V)_i = B V_i + eps_u g_i^{-1/2} sum_f c_f (U_i - U_j), so the B terms cancel in b except
// when the remainder is switched off (R = 0, b = -L V).
template <typename T>
__global__ void k_sec2_first(const int* __restrict__ idx, const int* __restrict__ count, ModelC<T> mc, KrylovOp<T> op,
                             const T* __restrict__ sg, const T* __restrict__ U, const T* __restrict__ w,
                             const double* __restrict__ scal, double hvol, T* __restrict__ R0, T* __restrict__ b) {
  const int M = *count;
  const T mass = (T)(hvol * scal[S_MASS]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int p = idx[i];
    const T s = sg[i], u = U[p];
    T lap = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int j = op.v.nb[f * op.v.cap + i];
      lap += op.v.c[f * op.v.cap + i] * (u - U[idx[j]]);
    }
    const T nl = sec2_nl(mc, s, u, w[p], mass);
    const T BV = mc.B2 * s * u;
    R0[i] = mc.linear_only ? (T)0 : BV + nl;
    b[i] = (mc.linear_only ? -BV : nl) - mc.eps_u * op.isg[i] * lap;
  }
}

// Corrector right-hand side: d = R_phi(U~) - R0 at the band nodes.
template <typename T>
__global__ void k_sec2_second(const int* __restrict__ idx, const int* __restrict__ count, ModelC<T> mc,
                              const T* __restrict__ sg, const T* __restrict__ Ut, const T* __restrict__ w,
                              const double* __restrict__ scal, double hvol, const T* __restrict__ R0,
                              T* __restrict__ d) {
  const int M = *count;
  const T mass = (T)(hvol * scal[S_MASS]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int p = idx[i];
    const T s = sg[i], u = Ut[p];
    const T r = mc.linear_only ? (T)0 : mc.B2 * s * u + sec2_nl(mc, s, u, w[p], mass);
    d[i] = r - R0[i];
  }
}

// v = base + sum_{k < m} y_k V_k at the band nodes (base = g^{1/2} U_in when `base` is null);
// vt_out (nullable) keeps v, U_out = v / g^{1/2} at the band nodes.
template <typename T>
__global__ void k_krylov_finish(const int* __restrict__ idx, const int* __restrict__ count, const T* __restrict__ V,
                                int ld, const double* __restrict__ y, int m, const T* __restrict__ base,
                                const T* __restrict__ sg, const T* __restrict__ U_in, T* __restrict__ vt_out,
                                T* __restrict__ U_out) {
  const int M = *count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int p = idx[i];
    double v = base ? (double)base[i] : (double)sg[i] * (double)U_in[p];
    for (int k = 0; k < m; ++k) v += y[k] * (double)V[(size_t)k * ld + i];
    if (vt_out) vt_out[i] = (T)v;
    U_out[p] = (T)(v / (double)sg[i]);
  }
}

// ---- host side: phi_j of the small symmetric tridiagonal Lanczos matrix -----------------

// phi_0 .. phi_3 at real z >= 0 with phi_0(z) = e^{-z}, phi_{k+1}(z) = (1/k! - phi_k(z))/z
// (Sec. 2.2's convention): the series sum_n (-z)^n/(n+k)! below 1, the recurrence above.
inline void phi_all(double z, double* p) {
  if (std::fabs(z) < 1.0) {
    double inv_kf = 1.0;                       // 1/k!
    for (int k = 0; k < 4; ++k) {
      if (k > 0) inv_kf /= k;
      double s = 0.0, zn = 1.0, c = inv_kf;    // c = 1/(n+k)!
      for (int n = 0; n < 24; ++n) {
        s += zn * c;
        zn *= -z;
        c /= (n + k + 1);
      }
      p[k] = s;
    }
    return;
  }
  p[0] = std::exp(-z);
  p[1] = -std::expm1(-z) / z;
  p[2] = (1.0 - p[1]) / z;
  p[3] = (0.5 - p[2]) / z;
}

// T = Q diag(lam) Q^T for the symmetric tridiagonal T (diagonal a[0..m-1], off-diagonal
// b[0..m-2]) by cyclic Jacobi rotations on the dense matrix; Q row-major m x m.
inline void tridiag_eig(int m, const double* a, const double* b, std::vector<double>& lam, std::vector<double>& Q) {
  std::vector<double> A((size_t)m * m, 0.0);
  Q.assign((size_t)m * m, 0.0);
  double scale = 0.0;
  for (int i = 0; i < m; ++i) {
    A[(size_t)i * m + i] = a[i];
    Q[(size_t)i * m + i] = 1.0;
    scale = std::max(scale, std::fabs(a[i]));
    if (i + 1 < m) {
      A[(size_t)i * m + i + 1] = A[(size_t)(i + 1) * m + i] = b[i];
      scale = std::max(scale, std::fabs(b[i]));
    }
  }
  lam.resize(m);
  for (int sweep = 0; sweep < 60 && scale > 0.0; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) off = std::max(off, std::fabs(A[(size_t)p * m + q]));
    if (off <= 1e-17 * scale) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[(size_t)p * m + q];
        if (std::fabs(apq) <= 1e-300) continue;
        // rotation angle that zeroes A[p][q]: t = tan(theta), the smaller root
        const double th = (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {
          const double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
          A[(size_t)k * m + p] = c * akp - s * akq;
          A[(size_t)k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {
          const double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
          A[(size_t)p * m + k] = c * apk - s * aqk;
          A[(size_t)q * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double qkp = Q[(size_t)k * m + p], qkq = Q[(size_t)k * m + q];
          Q[(size_t)k * m + p] = c * qkp - s * qkq;
          Q[(size_t)k * m + q] = s * qkp + c * qkq;
        }
      }
  }
  for (int i = 0; i < m; ++i) lam[i] = A[(size_t)i * m + i];
}

// y = phi_j(tau T_m) e_1 (length m) and the estimate |e_m^T phi_{j+1}(tau T_m) e_1| of the
// first term the Krylov space of dimension m leaves out.
inline double krylov_coeffs(int m, const double* alpha, const double* beta, double tau, int j, std::vector<double>& y) {
  std::vector<double> lam, Q;
  tridiag_eig(m, alpha, beta, lam, Q);
  y.assign(m, 0.0);
  double tail = 0.0;
  for (int k = 0; k < m; ++k) {
    double p[4];
    phi_all(tau * lam[k], p);
    const double q0 = Q[(size_t)0 * m + k];
    for (int r = 0; r < m; ++r) y[r] += Q[(size_t)r * m + k] * p[j] * q0;
    tail += Q[(size_t)(m - 1) * m + k] * p[j + 1] * q0;
  }
  return std::fabs(tail);
}

}  // namespace etd
