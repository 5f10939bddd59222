// rve_project_noalloc: the float64 projection G : A for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: plugins of host programs that
// own every device allocation themselves and hand out only their own
// buffers, or real-time paths where an allocation (and the implicit device
// synchronisation it may bring) is not allowed.  For them this file keeps
// the scratch of the projection -- the float64 half spectrum of the nine
// components and the twiddle tables -- in one fixed device array that lives
// as long as the library is loaded.  Every GPU that loads the library holds
// RVE_NOALLOC_SCRATCH_BYTES of it until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/rve.h"
#include "kernels.h"

bool rve_internal_make_geom(int nx, int ny, int nz, GridGeom* g);

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[RVE_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
bool g_kernels_ready[kMaxDevices] = {};

// Per-device set-up, done once per device with that device current and under
// the lock: the device address of the scratch array (in host code the array's
// name only stands for a host-side shadow, so the address is looked up with
// cudaGetSymbolAddress) and the shared-memory attributes of the transform
// kernels.  Later calls only read the cached address.
int device_setup(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RVE_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return RVE_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RVE_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  if (!g_kernels_ready[dev]) {
    if (fft_kernels_init() != cudaSuccess) return RVE_ERR_CUDA;
    g_kernels_ready[dev] = true;
  }
  *out = g_scratch_addr[dev];
  return RVE_OK;
}

// tw[k] = exp(-2 pi i k / N) for the three axes, in float64.
__global__ void k_noalloc_twiddles(cplx<double>* tw, int nx, int ny, int nz) {
  const int tot = nx + ny + nz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
    int k = i, n = nx;
    if (k >= nx) {
      k -= nx;
      n = ny;
      if (k >= ny) {
        k -= ny;
        n = nz;
      }
    }
    double s, c;
    sincospi(2.0 * (double)k / (double)n, &s, &c);
    tw[i] = {c, -s};
  }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int rve_project_noalloc(int nx, int ny, int nz, const double* A, double* out,
                                   void* stream) {
  if (!A || !out) return RVE_ERR_INVALID;
  GridGeom g;
  if (!rve_internal_make_geom(nx, ny, nz, &g)) return RVE_ERR_INVALID;
  const size_t tw_bytes = align256(sizeof(cplx<double>) * ((size_t)nx + ny + nz));
  const size_t spec_bytes = sizeof(cplx<double>) * 9 * g.sstride;
  if (tw_bytes + spec_bytes > (size_t)RVE_NOALLOC_SCRATCH_BYTES) return RVE_ERR_NOMEM;
  void* base = nullptr;
  int rc = device_setup(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cplx<double>* tw = reinterpret_cast<cplx<double>*>(base);
  cplx<double>* spec = reinterpret_cast<cplx<double>*>(reinterpret_cast<char*>(base) + tw_bytes);
  // every call rewrites the twiddles and every spectrum entry it later reads,
  // so nothing left in the shared array by an earlier call is used
  k_noalloc_twiddles<<<4, 256, 0, s>>>(tw, nx, ny, nz);
  Twiddles<double> t{tw, tw + nx, tw + nx + ny};
  TangentView<double> plain{};
  plain.mode = 0;
  launch_zfwd<double>(g, SRC_FIELD, plain, A, nullptr, nullptr, nullptr, nullptr, nullptr, spec, t,
                      s);
  launch_fft_y<double>(g, false, spec, nullptr, t, s);
  launch_fft_x_proj<double>(g, 1.0 / (double)g.n, spec, nullptr, t, s);
  launch_fft_y<double>(g, true, spec, nullptr, t, s);
  launch_zinv<double, double>(g, OUT_PLAIN, spec, out, nullptr, nullptr, nullptr, nullptr, nullptr,
                              nullptr, t, s);
  if (cudaGetLastError() != cudaSuccess) return RVE_ERR_CUDA;
  return RVE_OK;
}
