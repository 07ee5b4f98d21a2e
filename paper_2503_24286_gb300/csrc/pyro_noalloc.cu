// Net production rates without any device allocation.
//
// Some callers cannot call cudaMalloc when they evaluate the chemistry: a flow
// solver whose memory pool already holds the whole device (a new allocation
// would fail or force the pool to give memory back), or a time-step loop that
// must not take cudaMalloc's implicit device-wide synchronisation.  For them,
// this entry point stages the caller's arrays and the Newton failure counter
// through one fixed scratch array that lives in this file as a static device
// variable.  Its module is loaded, and its memory taken, when the first
// mechanism handle is loaded on a GPU (pyro_mech_load calls
// noalloc_prepare_device, which also looks up the array's device address), and
// every GPU that loads a handle keeps it until the process exits.  The entry
// point itself calls no cudaMalloc, cudaFree or any other allocating routine.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "pyro.h"
#include "pyro_internal.h"

namespace {

// The scratch: staged rho, T-or-e, Y, T_out, omega and the failure counter.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PYRO_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device.  The host-side name
// g_noalloc_scratch is only a stand-in for the symbol, not a device address, so
// the address is queried once per device (with that device current) and kept.
int scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return pyro::internal_fail(PYRO_ECUDA, "pyro_net_production_rates_noalloc: no current CUDA device");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      std::string m = std::string("pyro_net_production_rates_noalloc: cudaGetSymbolAddress failed: ") +
                      cudaGetErrorString(e);
      return pyro::internal_fail(PYRO_ECUDA, m.c_str());
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PYRO_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

namespace pyro {
int noalloc_prepare_device() {
  void* p = nullptr;
  return scratch_address(&p);
}
}  // namespace pyro

extern "C" int pyro_net_production_rates_noalloc(const pyro_mech* mech, int64_t n, const double* rho,
                                                 const double* T_or_e, int input_is_energy,
                                                 const double* Y, double* T_out, double* omega_out,
                                                 void* stream) {
  if (!mech || n < 0 || (n > 0 && (!rho || !T_or_e || !Y || !omega_out)))
    return pyro::internal_fail(PYRO_EINVAL, "pyro_net_production_rates_noalloc: bad arguments");
  if (input_is_energy && !T_out)
    return pyro::internal_fail(PYRO_EINVAL, "pyro_net_production_rates_noalloc: T_out is required when input_is_energy != 0");
  if (n == 0) return PYRO_OK;
  if (int rc = pyro::internal_check_device(mech)) return rc;
  const size_t N = (size_t)pyro::internal_n_species(mech);
  const size_t s1 = (size_t)n * sizeof(double);
  // layout: counter | rho | T_or_e | Y | T_out | omega, each 256-byte aligned
  const size_t off_rho = 256, off_t = off_rho + align256(s1), off_y = off_t + align256(s1);
  const size_t off_to = off_y + align256(N * s1), off_w = off_to + align256(s1);
  const size_t total = off_w + align256(N * s1);
  if ((uint64_t)n > (uint64_t)PYRO_NOALLOC_SCRATCH_BYTES || total > (size_t)PYRO_NOALLOC_SCRATCH_BYTES) {
    size_t per = (2 * N + 3) * sizeof(double);
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "pyro_net_production_rates_noalloc: n = %lld states need %zu bytes of scratch; the fixed "
                  "scratch holds %u bytes (at most about %zu states of this %zu-species mechanism per call)",
                  (long long)n, total, (unsigned)PYRO_NOALLOC_SCRATCH_BYTES,
                  (size_t)(PYRO_NOALLOC_SCRATCH_BYTES - 6 * 256) / per, N);
    return pyro::internal_fail(PYRO_EINVAL, msg);
  }
  void* base = nullptr;
  if (int rc = scratch_address(&base)) return rc;
  unsigned char* b = (unsigned char*)base;
  cudaStream_t s = (cudaStream_t)stream;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s) == cudaSuccess;
  };
  // the scratch keeps the previous call's contents: the failure counter must start at zero
  if (cudaMemsetAsync(b, 0, sizeof(unsigned long long), s) != cudaSuccess ||
      !cp(b + off_rho, rho, s1) || !cp(b + off_t, T_or_e, s1) || !cp(b + off_y, Y, N * s1))
    return pyro::internal_fail(PYRO_ECUDA, "pyro_net_production_rates_noalloc: copy into scratch failed");
  int rc = pyro::internal_launch_omega(mech, n, b + off_rho, b + off_t, input_is_energy, b + off_y,
                                       input_is_energy ? (void*)(b + off_to) : nullptr, b + off_w,
                                       (unsigned long long*)b, stream);
  if (rc) return rc;
  unsigned long long failed = 0;
  if (!cp(omega_out, b + off_w, N * s1) || (input_is_energy && !cp(T_out, b + off_to, s1)) ||
      !cp(&failed, b, sizeof failed) || cudaStreamSynchronize(s) != cudaSuccess)
    return pyro::internal_fail(PYRO_ECUDA, "pyro_net_production_rates_noalloc: copy out of scratch failed");
  if (failed) {
    std::string m = std::to_string(failed) + " point(s) did not converge in the Newton solve";
    return pyro::internal_fail(PYRO_ENOCONV, m.c_str());
  }
  return PYRO_OK;
}
