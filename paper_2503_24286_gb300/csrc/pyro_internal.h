// Internal (non-ABI) helpers shared between the runtime and other translation
// units of libpyro.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

struct pyro_mech;

namespace pyro {

// Number of species of a loaded mechanism.
int internal_n_species(const pyro_mech* h);

// PYRO_OK if h is a device handle whose device is current, else an error status
// (message set for pyro_last_error).
int internal_check_device(const pyro_mech* h);

// Set the calling thread's error message and return code.
int internal_fail(int code, const char* msg);

// Launch the net-production-rate kernel on device pointers, counting Newton
// failures into `fail` (a device address).  Asynchronous on `stream`.
int internal_launch_omega(const pyro_mech* h, int64_t n, const void* rho, const void* T_or_e,
                          int input_is_energy, const void* Y, void* T_out, void* omega,
                          unsigned long long* fail, void* stream);

// Look up, on the current device, the address of the static scratch of
// pyro_net_production_rates_noalloc (pyro_noalloc.cu) and keep it.  Called by
// pyro_mech_load, so the scratch's module is loaded and its memory taken while
// loading a handle rather than inside a no-allocation call.
int noalloc_prepare_device();

// ---- learned initial guess (pyro_mlp.cu) ----
struct MlpState;
int mlp_n_params(int D);
int mlp_create(int D, MlpState** out);
void mlp_free(MlpState* s);
int mlp_set(MlpState* s, const double* params, const double* norm4);
int mlp_get(MlpState* s, double* params, double* norm4);
int mlp_grad(MlpState* s, int64_t n, int64_t start, int B, int N, const double* e, const double* Y,
             const double* T, double* loss_out, double* grad_out, cudaStream_t st);
int mlp_train(MlpState* s, int64_t n, int N, const double* e, const double* Y, const double* T, int epochs,
              int batch, double lr, unsigned seed, double* final_loss, cudaStream_t st);
int mlp_save(const MlpState* s, const char* path);
int mlp_load(MlpState* s, const char* path);
const void* mlp_device_bf16(const MlpState* s);
const float* mlp_device_params(const MlpState* s);
const float* mlp_host_norm(const MlpState* s);
bool mlp_ready(const MlpState* s);

}  // namespace pyro
