// ops.cuh -- spectral operators run inside pass B on the spectrum held in shared memory.
//
// Coefficient tables (built in FP64 on the host, Sec. 2.2 phi-functions of Sec. 3.2
// symbols): for every integer m = |k|^2 of the cubic box one row of 4 values (the fourth
// unused, so that one aligned vector load fetches a row)
//   tab [4m + 0..2] = phi0, tau phi1, tau phi2 at z = tau l^phi(lambda_m)
//   tabu[4m + 0..2] = phi0 - 1, tau phi1, tau phi2 at z = tau l^u(lambda_m)
// (phi0 - 1 = expm1(-z): the u-stage transforms the increment of G u, see OpUPred)
// with lambda_m = -(pi/X)^2 m.
//   tab [4m + 3]    = phi0 - 1 = expm1(-z) at z = tau l^phi (the increment form below)
//
// In the FP32-mixed form the carried phi spectrum is double-float (dcomplex, see df32.cuh)
// and the phi-stage advances it by increments: phi^{n+1}^ - phi^n^ is formed in FP32 (each
// term of it is accurate to its own rounding), added to the double-float spectrum, and
// inverse-transformed in FP32 into the increment of the double-float real-space phi.
#pragma once
#include "fft.cuh"

namespace etd {

// Stored-spectrum element of type S as the operator's working complex type C: the same
// value, or the nearest FP32 complex of a double-float one.
template <typename C, typename S> __device__ __forceinline__ C conv(const S& v) { return v; }
template <> __device__ __forceinline__ float2 conv<float2, dcomplex>(const dcomplex& v) {
  return float2{to_float(v.x), to_float(v.y)};
}

template <typename T> struct SpecConst {
  const T* tab;    // phi-stage rows, 4 values per m
  const T* tabu;   // u-stage rows, 4 values per m
  T inv_n;         // 1/(Nx Ny Nz): the inverse transform's factor
  T kscale;        // pi / X
  T ksq;           // (pi / X)^2
};

template <typename T> struct Row3 {
  T a, b, c;
};
__device__ __forceinline__ Row3<float> load_row(const float* t, int m) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(t) + m);
  return Row3<float>{v.x, v.y, v.z};
}
__device__ __forceinline__ Row3<double> load_row(const double* t, int m) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(t) + 2 * m);
  return Row3<double>{v.x, v.y, __ldg(t + 4 * m + 2)};
}
// The whole FP32 row: phi0 (high part), tau phi1, tau phi2, phi0 (low part).
__device__ __forceinline__ float4 load_row4(const float* t, int m) { return __ldg(reinterpret_cast<const float4*>(t) + m); }

template <typename T, typename C>
__device__ __forceinline__ C deriv_mult(int o, C v, const Wave& w, const SpecConst<T>& k) {
  // o = 0: identity, 1: Laplacian (lambda), 2..4: d/dx, d/dy, d/dz (i k, Nyquist -> 0)
  if (o == 0) return cscale(v, k.inv_n);
  if (o == 1) return cscale(v, -k.ksq * (T)w.m * k.inv_n);
  const int s = (o == 2) ? w.sx : (o == 3 ? w.sy : w.sz);
  const T f = k.kscale * (T)s * k.inv_n;
  return C{-f * v.y, f * v.x};
}

// Forward only: store the spectrum (plan layout).
template <typename T> struct OpStore {
  using C = typename Cplx<T>::type;
  __device__ const void* pre() const { return nullptr; }
  __device__ size_t pre_elem() const { return sizeof(C); }
  static constexpr int NI = 1;
  int nout;
  C* spec;
  __device__ void combine(int, long long ge, const Wave&, C& s0, C&) const { spec[ge] = s0; }
  __device__ C out(int, C v, const Wave&) const { return v; }
};

// Load a stored spectrum and emit multipliers of it (identity, Laplacian, gradient).
// `sel` lists the outputs (codes of deriv_mult).
template <typename T, typename S = typename Cplx<T>::type> struct OpDeriv {
  using C = typename Cplx<T>::type;
  __device__ const void* pre() const { return nullptr; }
  __device__ size_t pre_elem() const { return sizeof(C); }
  static constexpr int NI = 0;
  int nout;
  int sel[5];
  const S* spec;
  SpecConst<T> k;
  __device__ void combine(int, long long ge, const Wave&, C& s0, C&) const { s0 = conv<C>(spec[ge]); }
  __device__ C out(int o, C v, const Wave& w) const { return deriv_mult<T>(sel[o], v, w, k); }
};

// phi-stage predictor (Sec. 3.3): R1^ = FFT(R_rest) + kappa/(mu eps^2) lambda FFT(W'-A1 phi),
// phi~^ = phi0 phi^n^ + tau phi1 R1^.  RK2 stores S = phi~^ - tau phi2 R1^ (so that the
// corrector is S + tau phi2 R1(phi~)^); ETD1 overwrites phi^ with phi~^.
template <typename T> struct OpPhiPred {
  using C = typename Cplx<T>::type;
  __device__ const void* pre() const { return spec_phi; }  // stored spectrum read in combine
  __device__ size_t pre_elem() const { return sizeof(C); }
  static constexpr int NI = 2;
  int nout;
  int sel[5];
  C* spec_phi;     // phi^n^ (ETD1: overwritten with phi^{n+1}^)
  C* spec_S;       // RK2 only
  int rk2;
  T c_lap;         // kappa / (mu eps_phi^2)
  SpecConst<T> k;
  __device__ void combine(int, long long ge, const Wave& w, C& s0, C& s1) const {
    const T lam = -k.ksq * (T)w.m;
    const C r1 = C{s0.x + c_lap * lam * s1.x, s0.y + c_lap * lam * s1.y};
    const Row3<T> c = load_row(k.tab, w.m);
    const T a0 = c.a, a1 = c.b;
    const C v = spec_phi[ge];
    const C pt = C{a0 * v.x + a1 * r1.x, a0 * v.y + a1 * r1.y};
    if (rk2) {
      const T a2 = c.c;
      spec_S[ge] = C{pt.x - a2 * r1.x, pt.y - a2 * r1.y};
    } else {
      spec_phi[ge] = pt;
    }
    s0 = pt;
  }
  __device__ C out(int o, C v, const Wave& w) const { return deriv_mult<T>(sel[o], v, w, k); }
};

// phi-stage corrector: phi^{n+1}^ = S + tau phi2 R1(phi~)^ ; stored and emitted.
template <typename T> struct OpPhiCorr {
  using C = typename Cplx<T>::type;
  __device__ const void* pre() const { return spec_S; }  // stored spectrum read in combine
  __device__ size_t pre_elem() const { return sizeof(C); }
  static constexpr int NI = 2;
  int nout;
  C* spec_phi;
  const C* spec_S;
  T c_lap;
  SpecConst<T> k;
  __device__ void combine(int, long long ge, const Wave& w, C& s0, C& s1) const {
    const T lam = -k.ksq * (T)w.m;
    const C r1 = C{s0.x + c_lap * lam * s1.x, s0.y + c_lap * lam * s1.y};
    const T a2 = __ldg(k.tab + 4 * w.m + 2);
    const C S = spec_S[ge];
    const C p = C{S.x + a2 * r1.x, S.y + a2 * r1.y};
    spec_phi[ge] = p;
    s0 = p;
  }
  __device__ C out(int, C v, const Wave&) const { return cscale(v, k.inv_n); }
};

// phi-stage predictor on the double-float spectrum (FP32-mixed form), as increments:
//   D1 = phi~^ - phi^n^ = (phi0 - 1) phi^n^ + tau phi1 R1^   (FP32; phi0 - 1 from tab[4m+3])
//   phi~^ = phi^n^ + D1 (double-float, rounded for the FP32 outputs phi~, Delta phi~, grad phi~)
//   RK2: S' = D1 - tau phi2 R1^ stored (FP32), so that phi^{n+1}^ - phi^n^ = S' + tau phi2 R1(phi~)^;
//   ETD1: phi^{n+1}^ = phi~^ stored, and the single output is the increment D1 / N.
struct OpPhiPredInc {
  using C = float2;
  __device__ const void* pre() const { return spec_phi; }  // stored spectrum read in combine
  __device__ size_t pre_elem() const { return sizeof(dcomplex); }
  static constexpr int NI = 2;
  int nout;
  int sel[5];
  dcomplex* spec_phi;
  C* spec_S;
  int rk2;
  float c_lap;
  SpecConst<float> k;
  __device__ void combine(int, long long ge, const Wave& w, C& s0, C& s1) const {
    const float lam = -k.ksq * (float)w.m;
    const C r1 = C{s0.x + c_lap * lam * s1.x, s0.y + c_lap * lam * s1.y};
    const float4 c = load_row4(k.tab, w.m);
    const dcomplex v = spec_phi[ge];
    const C d1 = C{c.w * v.x.hi + c.y * r1.x, c.w * v.y.hi + c.y * r1.y};
    const dcomplex pt{add_f(v.x, d1.x), add_f(v.y, d1.y)};
    if (rk2) {
      spec_S[ge] = C{d1.x - c.z * r1.x, d1.y - c.z * r1.y};
      s0 = conv<C>(pt);
    } else {
      spec_phi[ge] = pt;
      s0 = d1;
    }
  }
  __device__ C out(int o, C v, const Wave& w) const { return deriv_mult<float>(sel[o], v, w, k); }
};

// phi-stage corrector on the double-float spectrum: D = S' + tau phi2 R1(phi~)^ is
// phi^{n+1}^ - phi^n^; the spectrum takes phi^n^ + D (double-float) and the output is D / N.
struct OpPhiCorrInc {
  using C = float2;
  __device__ const void* pre() const { return spec_phi; }  // stored spectrum read in combine
  __device__ size_t pre_elem() const { return sizeof(dcomplex); }
  static constexpr int NI = 2;
  int nout;
  dcomplex* spec_phi;
  const C* spec_S;
  float c_lap;
  SpecConst<float> k;
  __device__ void combine(int, long long ge, const Wave& w, C& s0, C& s1) const {
    const float lam = -k.ksq * (float)w.m;
    const C r1 = C{s0.x + c_lap * lam * s1.x, s0.y + c_lap * lam * s1.y};
    const float a2 = __ldg(k.tab + 4 * w.m + 2);
    const C Sv = spec_S[ge];
    const C d = C{Sv.x + a2 * r1.x, Sv.y + a2 * r1.y};
    const dcomplex v = spec_phi[ge];
    spec_phi[ge] = dcomplex{add_f(v.x, d.x), add_f(v.y, d.y)};
    s0 = d;
  }
  __device__ C out(int, C v, const Wave&) const { return cscale(v, k.inv_n); }
};

// u-stage predictor as an increment: D~^ = GU~^ - FFT(G u^n) = (phi0 - 1) FFT(G u^n) + tau phi1 R2^,
// so that GU~ = G u^n + IFFT(D~^) (EpiRecover adds G u^n back); RK2 stores S = D~^ - tau phi2 R2^.
template <typename T> struct OpUPred {
  using C = typename Cplx<T>::type;
  __device__ const void* pre() const { return nullptr; }
  __device__ size_t pre_elem() const { return sizeof(C); }
  static constexpr int NI = 2;
  int nout;
  C* spec_S;
  int rk2;
  SpecConst<T> k;
  __device__ void combine(int, long long ge, const Wave& w, C& s0, C& s1) const {
    const Row3<T> c = load_row(k.tabu, w.m);
    const C p = C{c.a * s0.x + c.b * s1.x, c.a * s0.y + c.b * s1.y};
    if (rk2) spec_S[ge] = C{p.x - c.c * s1.x, p.y - c.c * s1.y};
    s0 = p;
  }
  __device__ C out(int, C v, const Wave&) const { return cscale(v, k.inv_n); }
};

// u-stage corrector: GU^{n+1}^ - FFT(G u^n) = S + tau phi2 R2(U~)^.
template <typename T> struct OpUCorr {
  using C = typename Cplx<T>::type;
  __device__ const void* pre() const { return spec_S; }  // stored spectrum read in combine
  __device__ size_t pre_elem() const { return sizeof(C); }
  static constexpr int NI = 1;
  int nout;
  const C* spec_S;
  SpecConst<T> k;
  __device__ void combine(int, long long ge, const Wave& w, C& s0, C&) const {
    const T b2 = __ldg(k.tabu + 4 * w.m + 2);
    const C S = spec_S[ge];
    s0 = C{S.x + b2 * s0.x, S.y + b2 * s0.y};
  }
  __device__ C out(int, C v, const Wave&) const { return cscale(v, k.inv_n); }
};

// Standard-layout half spectrum [kz][ky][kx] in/out (operator entry points).
template <typename T> struct OpToStd {
  using C = typename Cplx<T>::type;
  __device__ const void* pre() const { return nullptr; }
  __device__ size_t pre_elem() const { return sizeof(C); }
  static constexpr int NI = 1;
  int nout;
  C* dst;
  int ny, nxh;
  __device__ void combine(int, long long, const Wave& w, C& s0, C&) const {
    dst[((long long)w.kz * ny + w.ky) * nxh + w.kx] = s0;
  }
  __device__ C out(int, C v, const Wave&) const { return v; }
};

template <typename T> struct OpFromStd {
  using C = typename Cplx<T>::type;
  __device__ const void* pre() const { return nullptr; }
  __device__ size_t pre_elem() const { return sizeof(C); }
  static constexpr int NI = 0;
  int nout;
  const C* src;
  int ny, nxh;
  T inv_n;
  __device__ void combine(int, long long, const Wave& w, C& s0, C&) const {
    s0 = src[((long long)w.kz * ny + w.ky) * nxh + w.kx];
  }
  __device__ C out(int, C v, const Wave&) const { return cscale(v, inv_n); }
};

}  // namespace etd
