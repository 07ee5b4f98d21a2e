// Internal (non-ABI) helpers shared between the runtime and other translation
// units of libpyro.
#pragma once

#include <stdint.h>

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

}  // namespace pyro
