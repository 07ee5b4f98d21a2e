// Emitter of the warp-per-state kernels (one warp per state, lanes splitting the
// species and the reactions) for large mechanisms.
#pragma once

#include <map>
#include <string>

#include "pyro_emit.h"
#include "pyro_mech.h"

namespace pyro {

struct WarpEmit {
  // "wfwd": pyro_omega_warp, "wjvp": pyro_jvp_warp, "wvjp": pyro_vjp_warp,
  // "wjac": pyro_jacobian_cta, "wjad": pyro_jacobian_adiabatic_cta
  std::map<std::string, std::string> sources;
  std::map<std::string, double> stats;
  std::map<std::string, int> wpb;               // warps (states) per block of each kernel
  std::map<std::string, int> smem;              // dynamic shared memory per block of each kernel
  int warps_per_block = 8;                      // of the forward kernel
  int smem_bytes = 0;
};

// Limits of the emitted tables (packed indices): species, reactions, and the
// production-rate segments (species + 32).
constexpr int kWarpMaxSpecies = 1022;
constexpr int kWarpMaxReactions = 65535;

// Blocks (consecutive states) per thread-block cluster of the block-per-state
// Jacobian kernels: the dense write pass of a cluster covers its states together,
// four lanes filling one 32-byte sector of the output.  Grids are multiples of it.
constexpr int kJacCluster = 4;

// Whether the warp-per-state kernels cover the mechanism: the limits above, at
// most three factors on each side of a reaction (packed factor lists; net
// stoichiometric coefficients -3..3), and one NASA-7 T_mid shared by all species
// (one range choice per state).  Otherwise *why says what is not met.
bool warp_supported(const Mechanism& m, std::string* why);

WarpEmit emit_warp_units(const Mechanism& m, const EmitOptions& opt);

}  // namespace pyro
