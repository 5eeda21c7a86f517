// etd_static.cu -- the forward FFT without any device allocation.
//
// Who needs this: a caller whose device memory is owned by someone else (a host
// application that hands out all device memory from its own pool, or runs with a fixed,
// pre-budgeted footprint), and a caller on a latency-critical path where cudaMalloc or
// cudaFree may implicitly synchronise the device.  Such callers cannot create a plan,
// because etd_plan allocates its workspace.  This entry point takes the caller's input and
// output buffers and keeps its own scratch (the pass-A -> pass-B intermediate spectrum and
// the twiddle tables) in one file-scope device array that every GPU loading the library
// holds until the process exits.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include "etd.h"
#include "fft.cuh"
#include "kernels.cuh"
#include "ops.cuh"

namespace etd {
void set_last_error(const std::string& msg);
}

#define ETD_STATIC_SCRATCH_BYTES (8u << 20)

// Shared by every call on a device; contents persist between calls.
static __device__ __align__(256) unsigned char etd_static_scratch[ETD_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// The host-side name of etd_static_scratch is not a device address.  Look the address up
// once per device, with that device current, and hand it to the kernels.
etd_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    etd::set_last_error("device ordinal out of range for the static scratch table");
    return ETD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, etd_static_scratch);
    if (e != cudaSuccess || !p) {
      etd::set_last_error(std::string("cudaGetSymbolAddress(etd_static_scratch): ") + cudaGetErrorString(e));
      return ETD_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return ETD_OK;
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// w_N^e = exp(-2 pi i e / N) written into the scratch area on every call.
template <typename C> __global__ void k_twiddles(C* tw, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * e / n, &s, &c);
    tw[e].x = (decltype(tw[e].x))c;
    tw[e].y = (decltype(tw[e].y))(-s);
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Scratch bytes: the intermediate spectrum, then the three twiddle tables.
size_t scratch_bytes(int dim, const int* n, size_t csize) {
  const size_t nz = dim == 2 ? 1 : (size_t)n[2];
  const size_t nhat = (size_t)(n[0] / 2 + 1) * n[1] * nz;
  return align256(csize * nhat) + align256(csize * n[0]) + align256(csize * n[1]) + align256(csize * nz);
}

template <typename T>
etd_status run(int dim, const int* n, const void* field, void* half, cudaStream_t st, unsigned char* scratch) {
  using C = typename etd::Cplx<T>::type;
  etd::Geo g{};
  const int nx = n[0], ny = n[1], nz = dim == 2 ? 1 : n[2];
  g.dim = dim;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.nxh = nx / 2 + 1;
  g.n = (long long)nx * ny * nz;
  g.nhat = (long long)g.nxh * ny * nz;
  const size_t inter = align256(sizeof(C) * (size_t)g.nhat);
  // same tile rule as a plan
  size_t smemA = 0, smemB1 = 0;
  if (!etd::choose_tiles(g, sizeof(C), smemA, smemB1)) {
    etd::set_last_error("grid not supported by the two-pass FFT tiles");
    return ETD_EINVAL;
  }
  const size_t smemB = smemB1;  // one operand tile (forward only)

  C* I = reinterpret_cast<C*>(scratch);
  C* twx = reinterpret_cast<C*>(scratch + inter);
  C* twy = reinterpret_cast<C*>(scratch + inter + align256(sizeof(C) * nx));
  C* twz = reinterpret_cast<C*>(scratch + inter + align256(sizeof(C) * nx) + align256(sizeof(C) * ny));
  k_twiddles<C><<<4, 256, 0, st>>>(twx, nx);
  k_twiddles<C><<<4, 256, 0, st>>>(twy, ny);
  k_twiddles<C><<<4, 256, 0, st>>>(twz, nz);

  auto ka = etd::passA_fwd<T, etd::ProLoad<T>>;
  auto kb = etd::passB<T, etd::OpToStd<T>>;
  int dev = 0, optin = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (ce != cudaSuccess) {
    etd::set_last_error(std::string("shared-memory limit query: ") + cudaGetErrorString(ce));
    return ETD_ECUDA;
  }
  if ((size_t)optin < smemA || (size_t)optin < smemB) {
    etd::set_last_error("grid needs " + std::to_string(std::max(smemA, smemB)) + " bytes of shared memory per block, " +
                        "the device allows " + std::to_string(optin));
    return ETD_EINVAL;
  }
  if (smemA > 48 * 1024) ce = cudaFuncSetAttribute((const void*)ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemA);
  if (ce == cudaSuccess && smemB > 48 * 1024)
    ce = cudaFuncSetAttribute((const void*)kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemB);
  if (ce != cudaSuccess) {
    etd::set_last_error(std::string("cudaFuncSetAttribute(MaxDynamicSharedMemorySize): ") + cudaGetErrorString(ce));
    return ETD_ECUDA;
  }
  CUtensorMap none;
  std::memset(&none, 0, sizeof(none));
  const etd::PassAIn plain{0, 0u, 0, nullptr, 0};  // direct stores (no tensor map, no wait)
  ka<<<(nz / g.ZB) * g.Y1, ETD_PASSA_THREADS, smemA, st>>>(g, etd::ProLoad<T>{static_cast<const T*>(field)}, I, twx, twy,
                                                           none, plain);
  etd::OpToStd<T> op{0, static_cast<C*>(half), g.ny, g.nxh};
  etd::OutP<C> outs{};
  const int nkb = (g.nxh + g.KB - 1) / g.KB;
  kb<<<nkb * g.Y2, ETD_PASSB_THREADS, smemB, st>>>(g, op, I, nullptr, outs, twy, twz);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    etd::set_last_error(std::string("launch: ") + cudaGetErrorString(e));
    return ETD_ECUDA;
  }
  return ETD_OK;
}

}  // namespace

extern "C" etd_status etd_fft_forward_noalloc(int dim, const int* n, int precision, const void* field,
                                              void* half_spectrum, void* cuda_stream) {
  if (!n || !field || !half_spectrum) {
    etd::set_last_error("NULL argument");
    return ETD_EINVAL;
  }
  if (dim != 2 && dim != 3) {
    etd::set_last_error("dim must be 2 or 3");
    return ETD_EINVAL;
  }
  for (int d = 0; d < 2; ++d)
    if (!pow2(n[d]) || n[d] < 8 || n[d] > 256) {
      etd::set_last_error("Nx, Ny must be powers of two in [8, 256]");
      return ETD_EINVAL;
    }
  if (dim == 3 && (!pow2(n[2]) || n[2] < 8 || n[2] > 256)) {
    etd::set_last_error("Nz must be a power of two in [8, 256]");
    return ETD_EINVAL;
  }
  if (precision != ETD_FP64 && precision != ETD_FP32_MIXED) {
    etd::set_last_error("unknown precision");
    return ETD_EINVAL;
  }
  const size_t need = scratch_bytes(dim, n, precision == ETD_FP64 ? 16 : 8);
  if (need > ETD_STATIC_SCRATCH_BYTES) {
    etd::set_last_error("grid needs " + std::to_string(need) + " bytes of scratch; the static scratch holds " +
                        std::to_string(ETD_STATIC_SCRATCH_BYTES) + " (half spectrum plus twiddles must fit)");
    return ETD_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    etd::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return ETD_ECUDA;
  }
  void* scratch = nullptr;
  etd_status s = scratch_address(dev, &scratch);
  if (s != ETD_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  s = precision == ETD_FP64 ? run<double>(dim, n, field, half_spectrum, st, static_cast<unsigned char*>(scratch))
                            : run<float>(dim, n, field, half_spectrum, st, static_cast<unsigned char*>(scratch));
  if (s == ETD_OK) etd::set_last_error("");
  return s;
}
