// Emitter: mechanism -> mechanism-specialised CUDA C for sm_103a.
#pragma once

#include <map>
#include <string>

#include "pyro_mech.h"

namespace pyro {

struct EmitOptions {
  int block = 128;            // threads per block (one point per thread)
  int min_blocks = 2;         // __launch_bounds__ minimum resident blocks
  bool mixed_newton = true;   // FP32 Newton to ~1e-5, then FP64 Newton (else FP64 only)
  int deriv_block = 64;       // threads per block of the JVP / VJP / Jacobian kernels
  // large mechanisms: per-point species arrays in a global scratch instead of
  // shared memory (forward / derivative kernels), species accumulators in the
  // output arrays instead of registers
  bool gstore = false;
  bool dgstore = false;
  bool acc_mem = false;
  // Jacobian-type kernels: rows assembled by loops over emitted tables (per-row
  // reaction lists, per-reaction species partials) instead of straight-line code
  bool jac_table = false;
  // Crank-Nicolson unit: also emit the right-hand-side-only kernel of the chord iteration
  bool cn_residual = false;
  int exp_ops = 4;            // device exponential: 4 (default) or 2 FP64-pipe operations
  int warp_exp_ops = 2;       // the same for the warp-per-state kernels (their code is compact, so
                              // the 2-operation form does not outgrow the instruction cache)
  bool exp_call = false;      // one called body instead of inlining at every use
};

struct EmitResult {
  std::string source;                     // CUDA C of the forward kernels
  std::map<std::string, std::string> group_sources;   // "fwd", "jvp", "vjp", "jac", "jad", "cn"

  std::map<std::string, double> stats;    // static FP64-pipe op counts per point etc.
  int smem_dyn_bytes_omega = 0;           // dynamic shared memory of the omega kernel
  int smem_dyn_bytes_deriv = 0;           // dynamic shared memory of the derivative kernels
  int jac_slots = 0;                      // scratch doubles per point of the Jacobian kernel
  int smem_dyn_bytes_cn_solve = 0;        // dynamic shared memory of the Crank-Nicolson solve kernel
  int smem_dyn_bytes_transport = 0;       // dynamic shared memory of the transport kernel
  int smem_dyn_bytes_jac = 0;             // dynamic shared memory of the Jacobian-type kernels
  int cn_solve_warps = 4;                 // states (warps) per block of the Crank-Nicolson solve kernel
  // warp-per-state kernels ("wfwd", "wjvp", "wvjp"): states (warps) per block and
  // dynamic shared memory per block
  std::map<std::string, int> warp_wpb, smem_dyn_bytes_warp;
};

// Threads per block of the transport kernel (3 per-state arrays of N doubles in
// shared memory: 32-thread blocks fit 5 per SM for 53 species).
constexpr int kTransportBlock = 32;

// States per group of the Crank-Nicolson Newton-matrix layout [n/G][N^2][G]
// (also the warps per block of the batched solve).
constexpr int kCnGroup = 4;

EmitResult emit_module(const Mechanism& m, const EmitOptions& opt);

// The device-math header text (embedded at build time).
extern const char* kDeviceMathSource;

}  // namespace pyro
