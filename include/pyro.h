/* libpyro: GB300-native pointwise combustion thermochemistry (C ABI).
 *
 * The library evaluates, for millions of independent states, the
 * thermochemistry of a detailed kinetic mechanism as formulated in the
 * Pyrometheus paper (arXiv 2503.24286, Appendix A):
 *   - temperature from mixture internal energy by Newton iteration on two-range
 *     NASA-7 polynomials (Sec. A.3.1, Eq. int_energy, Eq. delta_temp, Eq. cv);
 *   - species thermodynamics (Sec. A.1, Eq. nasa_poly, Eq. nasa_poly_c, Eq. gibbs);
 *   - Arrhenius rate coefficients (Eq. rate_coeff) with third-body efficiencies
 *     and Troe falloff, equilibrium constants from Gibbs energies
 *     (Eq. equil_constants), mass-action rates of progress (Eq. reaction_rates)
 *     and net production rates (Eq. production_rates);
 *   - derivatives of the production rates (Eq. jacobian, Eq. chem_jacobian).
 *
 * Conventions for every entry point below:
 *   - Units: SI with kmol (rho kg/m^3, T K, e J/kg, omega kmol/(m^3 s), p Pa).
 *   - Arrays are FP64, structure-of-arrays with the point index fastest:
 *     Y[k*n + p] for species k, point p (the species-major layout of the
 *     paper's array inputs).  Per-point scalars are [n].
 *   - Pointers may be device pointers (CUDA global memory of the device the
 *     mechanism was loaded on) or host pointers.  With device pointers the call
 *     is asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  With host pointers (all array arguments of the call on the host)
 *     the library stages the data through its own device buffers, and the call
 *     returns after the results have been copied back.  Mixed host/device
 *     argument lists are rejected with PYRO_EINVAL.
 *   - The caller owns all arrays; the library owns the mechanism handle, the
 *     compiled module and its staging buffers.
 *   - Return value: PYRO_OK (0) or a negative status; argument checks are made
 *     before anything is launched.  pyro_last_error() gives the message of the
 *     calling thread's last failure.
 *   - n == 0 is a no-op that returns PYRO_OK.
 *   - A handle keeps per-handle work arrays (Jacobian partials, Crank-Nicolson
 *     work arrays, staging buffers of host-pointer calls) and compiles kernel
 *     groups on first use: calls on one handle from several host threads, or
 *     on several streams at once, must be serialised by the caller.  Separate
 *     handles are independent.
 */
#ifndef PYRO_H
#define PYRO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PYRO_OK 0
#define PYRO_EINVAL (-1)   /* bad argument (null pointer, n < 0, mixed host/device) */
#define PYRO_ECUDA (-2)    /* CUDA runtime/driver error */
#define PYRO_ECOMPILE (-3) /* NVRTC compilation of the emitted kernels failed */
#define PYRO_EMECH (-4)    /* mechanism file unreadable or fails validation */
#define PYRO_ENOCONV (-5)  /* Newton iteration did not converge for some points */
#define PYRO_ENOMLP (-6)   /* learned guess requested but no network is loaded */

typedef struct pyro_mech pyro_mech;

/* Load a mechanism file (text format "pyro-mech 1"), validate it (element
 * balance of every reaction, positive Arrhenius factors, NASA ranges, cp/R > 1,
 * Troe data), emit the mechanism-specialised CUDA C, compile it for sm_103a
 * with NVRTC (cached on disk by source hash) and load it on the current device.
 * options: NULL or "key=value;..." with keys
 *   block=<threads per block, default 128>
 *   newton=mixed|fp64   (mixed: FP32 Newton to |dT|<=1e-5 T, then FP64; fp64:
 *                        FP64 Newton from the initial guess as in Sec. A.3.1)
 *   cache=0|1           (on-disk cubin cache, default 1; dir $PYRO_CACHE_DIR)
 *   checked=0|1         (1: calls that run Newton synchronise and return
 *                        PYRO_ENOCONV if any point failed to converge)
 *   deriv_block=<threads per block of the derivative kernels, default 64>
 *   exp=4|2|4call|2call (device exponential: 4 FP64-pipe operations (default)
 *                        or 2 with the second-order terms in FP32 pairs; inlined
 *                        at every use, or one called body)
 *   warp_exp=2|4        (the exponential of the warp-per-state kernels: 2 FP64-pipe
 *                        operations (default; their code is compact) or 4)
 *   variant=thread|warp (net production rates: one thread per state with
 *                        mechanism-specialised straight-line code (default),
 *                        or one warp per state (pyro_net_production_rates,
 *                        pyro_jvp, pyro_vjp): the lanes split the species and
 *                        the reactions, in chunks of 32 reactions emitted for
 *                        the mechanism's reaction classes -- the faster form for
 *                        large mechanisms such as 160 species / 1100 reactions;
 *                        pyro_jacobian and pyro_jacobian_adiabatic then run one
 *                        block of 8 warps per state, in clusters of 4 blocks on
 *                        4 consecutive states, with no per-handle scratch).
 *                        variant=warp needs at most three factors on each side
 *                        of a reaction and one NASA-7 T_mid for all species
 *                        (PYRO_EINVAL otherwise)
 *   store=auto|shared|global  (where each thread keeps its state's species
 *                        arrays: shared memory, or -- automatic when they do
 *                        not fit, e.g. 160 species -- a library-owned global
 *                        scratch per kernel; calls of the same kernel on one
 *                        handle must then not overlap on the GPU)
 *   jac_rows=auto|inline|table (pyro_jacobian, pyro_jacobian_adiabatic,
 *                        pyro_cn_step: each row of the Jacobian as straight-line
 *                        code specialised to its species (inline), or as loops
 *                        over emitted per-row tables of reactions and species
 *                        partials (table; compiles in a fraction of the time for
 *                        large mechanisms); auto: table above 64 species)
 *   device=0|1          (0: parse, validate, emit and compile only; no CUDA
 *                        device is touched and nothing can be launched)
 *   cn_newton=full|chord (pyro_cn_step: Newton with the matrix re-assembled and
 *                        re-factored at every iterate (full, default, as in
 *                        Sec. A.3.2), or a chord iteration that keeps a
 *                        factorisation for cn_refresh iterations (the iterates in
 *                        between need only the right-hand side); same fixed
 *                        point and stop rule, more iterations: give max_newton
 *                        headroom)
 *   cn_refresh=<k>      (chord: re-assemble and re-factor at iterations 0, k, 2k, ...;
 *                        default 4)
 * On success *out receives a handle to free with pyro_mech_free. */
int pyro_mech_load(const char* mech_path, const char* options, pyro_mech** out);
void pyro_mech_free(pyro_mech* mech);

/* Sizes and molecular weights (host array of n_species doubles owned by the handle). */
int pyro_mech_info(const pyro_mech* mech, int* n_species, int* n_reactions,
                   const double** mol_weights);

/* Static per-point FP64-pipe operation counts of the emitted kernels and other
 * build facts, by name (e.g. "omega_fp64_flops_per_point").  PYRO_EINVAL if
 * the key is unknown. */
int pyro_mech_stat(const pyro_mech* mech, const char* key, double* value);

/* The emitted CUDA C source (owned by the handle). */
const char* pyro_mech_source(const pyro_mech* mech);

/* Density from the equation of state p = rho R T / W, W = (sum Y_k/W_k)^-1
 * (Sec. A.1 Eq. eos).  p, T: [n]; Y: [N][n]; rho: [n] out. */
int pyro_density(const pyro_mech* mech, int64_t n, const double* p, const double* T,
                 const double* Y, double* rho, void* stream);

/* Mixture internal energy e = sum_k Y_k (h_k - R T)/W_k (Sec. A.3.1 Eq. int_energy)
 * and, if cv != NULL, c_v = de/dT (Eq. cv).  T: [n]; Y: [N][n]; e, cv: [n] out. */
int pyro_internal_energy(const pyro_mech* mech, int64_t n, const double* T, const double* Y,
                         double* e, double* cv, void* stream);

/* Temperature from internal energy by Newton iteration (Sec. A.3.1 Eq. delta_temp).
 * e: [n]; Y: [N][n]; T_out: [n].
 * guess_mode 0: start from T_guess[p] if T_guess != NULL, else 1200 K.
 * guess_mode 1: start from the learned initial guess (BF16 MLP on the tensor
 *   cores, see pyro_mlp_train / pyro_mlp_load); PYRO_ENOMLP if none is
 *   loaded.  Points whose iteration from the guess fails restart from 1200 K
 *   (their count then includes the failed attempt plus max_iter + 1).
 * Stops when |dT| <= 1e-10 T, then takes one more step; at most 50 FP64 steps.
 * iters_out (nullable, int32 [n]): Newton steps taken, -1 where the stop rule
 * was not met (T_out then holds the last iterate).  Non-convergence is also
 * counted on the device; read it with pyro_nonconverged. */
int pyro_temperature(const pyro_mech* mech, int64_t n, const double* e, const double* Y,
                     const double* T_guess, int guess_mode, double* T_out, int32_t* iters_out,
                     void* stream);

/* Mixture enthalpy h = sum_k Y_k h_k / W_k (per unit mass; h_k from Sec. A.1
 * Eq. nasa_poly) and, if cp != NULL, c_p = dh/dT.  T: [n]; Y: [N][n]; h, cp: [n]
 * out. */
int pyro_enthalpy(const pyro_mech* mech, int64_t n, const double* T, const double* Y,
                  double* h, double* cp, void* stream);

/* Temperature from the mixture enthalpy (Sec. A.3.1: the Newton inversion with h
 * and c_p in place of e and c_v, for low-Mach and characteristic-boundary use).
 * h: [n]; Y: [N][n]; T_guess: nullable [n] (else 1200 K); T_out: [n];
 * iters_out: nullable int32 [n].  Stop rule, iteration cap, FP32-then-FP64
 * iteration and failure reporting as in pyro_temperature. */
int pyro_temperature_enthalpy(const pyro_mech* mech, int64_t n, const double* h, const double* Y,
                              const double* T_guess, double* T_out, int32_t* iters_out, void* stream);

/* Net production rates omega_k = sum_j nu_kj R_j (Sec. A.1 Eq. production_rates)
 * with R_j by the law of mass action (Eq. reaction_rates).
 * rho: [n]; T_or_e: [n] temperature, or internal energy if input_is_energy != 0
 * (then T is solved first as in pyro_temperature from 1200 K and written to
 * T_out, which must be non-NULL); Y: [N][n]; omega_out: [N][n]. */
int pyro_net_production_rates(const pyro_mech* mech, int64_t n, const double* rho,
                              const double* T_or_e, int input_is_energy, const double* Y,
                              double* T_out, double* omega_out, void* stream);

/* Compile and load derivative kernels ahead of their first use.  kernels:
 * NULL or "all" (jvp, vjp, jacobian), or a comma list of "jvp", "vjp",
 * "jacobian", "jacobian_adiabatic", "cn", "transport", "warp" (the
 * warp-per-state forward kernel).  The groups are
 * compiled in parallel host threads with NVRTC (cached on disk); without this
 * call each group is compiled on the first call that needs it. */
int pyro_mech_prepare(const pyro_mech* mech, const char* kernels);

/* Jacobian-vector product of the net production rates (forward mode):
 *   d_omega = (d omega/d rho) d_rho + (d omega/d T) d_T + sum_i (d omega/d Y_i) d_Y_i
 * at the state (rho, T, Y), differentiating Eq. production_rates with
 * Eq. reaction_rates, Eq. rate_coeff, Eq. equil_constants and the Troe form.
 * rho, T, d_rho, d_T: [n]; Y, d_Y: [N][n]; d_omega: [N][n] out. */
int pyro_jvp(const pyro_mech* mech, int64_t n, const double* rho, const double* T, const double* Y,
             const double* d_rho, const double* d_T, const double* d_Y, double* d_omega, void* stream);

/* Vector-Jacobian product (reverse mode, adjoint) of the same function:
 *   rho_bar = sum_k omega_bar_k d omega_k/d rho,  T_bar = sum_k omega_bar_k d omega_k/d T,
 *   Y_bar_i = sum_k omega_bar_k d omega_k/d Y_i.
 * omega_bar: [N][n]; rho_bar, T_bar: [n] out; Y_bar: [N][n] out.  The
 * per-reaction intermediates are recomputed, nothing is stored between passes. */
int pyro_vjp(const pyro_mech* mech, int64_t n, const double* rho, const double* T, const double* Y,
             const double* omega_bar, double* rho_bar, double* T_bar, double* Y_bar, void* stream);

/* Dense Jacobian for implicit integrators (Eq. jacobian, Eq. chem_jacobian):
 * J = d(Tdot, omega_1..omega_N)/d(T, Y_1..Y_N) at fixed rho, where Tdot is the
 * temperature rate of the adiabatic isochoric reactor (Sec. A.1 Eq. massfrac_ode
 * at fixed internal energy): Tdot = -sum_k (h_k - R T) omega_k / (rho c_v).
 * J: [(N+1)*(N+1)][n], entry (r, c) at J[(r*(N+1) + c)*n + p]; row 0 = Tdot,
 * row 1+k = omega_k; column 0 = T, column 1+i = Y_i.  The library keeps a
 * per-handle scratch buffer for the per-reaction partials (allocated on first
 * use, grown as needed; 8 B x pyro_mech_stat("jacobian_scratch_doubles_per_point")
 * x deriv_block (default 64) x the resident blocks: with the defaults ~0.6 GB for
 * 53 species, ~3 GB for 160 species and 1100 reactions): calls on one handle that use it (pyro_jacobian,
 * pyro_jacobian_adiabatic, pyro_cn_step) must not overlap on the GPU.  Handles
 * loaded with variant=warp use the block-per-state kernels instead, which keep
 * the partials in shared memory and need no scratch (their calls may overlap).
 * Needs all species to share one NASA-7 T_mid. */
int pyro_jacobian(const pyro_mech* mech, int64_t n, const double* rho, const double* T, const double* Y,
                  double* J, void* stream);

/* Chemical Jacobian of the source term at fixed density and internal energy
 * (Sec. A.3.2 Eq. chem_jacobian, with S_j = W_j omega_j of Eq. massfrac_ode):
 *   J_jk = dS_j/dY_k |_(rho, e) = W_j (d omega_j/dY_k + d omega_j/dT dT/dY_k),
 *   dT/dY_k = -e_k(T)/c_v  (Eq. int_energy, Eq. cv: T follows Y at fixed e).
 * T must be the temperature of (e, Y) (e.g. from pyro_temperature).
 * rho, T: [n]; Y: [N][n]; J: [N*N][n] out, entry (j, k) at J[(j*N + k)*n + p].
 * Columns sum to zero (mass conservation).  Shares the per-handle scratch of
 * pyro_jacobian.  Same mechanism restriction as pyro_jacobian. */
int pyro_jacobian_adiabatic(const pyro_mech* mech, int64_t n, const double* rho, const double* T,
                            const double* Y, double* J, void* stream);

/* One Crank-Nicolson step of the adiabatic isochoric reactor (Sec. A.3.2,
 * Eqs. crank_nicol_rhs, crank_nicol_newton_system, crank_nicol_newton_update,
 * crank_nicol_jac), reading Eq. massfrac_ode as dY/dt = S/rho at fixed (rho, e):
 *   F(Y) = Y - Y^m - dt/(2 rho) (S(Y) + S(Y^m)) = 0,
 * solved per state by Newton from Y^m with the matrix I - dt/(2 rho) J, J from
 * pyro_jacobian_adiabatic at each iterate and T re-solved from (e, Y) at each
 * iterate (e = e(T^m, Y^m)).  Stop once max_k |dY_k| <= tol, after one further
 * Newton step; at most max_newton steps.  The linear systems are solved by LU
 * with partial pivoting in FP32 on row-scaled matrices plus one step of
 * iterative refinement with an FP64 residual.
 * rho, T: [n] state at t^m; Y: [N][n]; T_out: [n] and Y_out: [N][n] at
 * t^m + dt (may alias T and Y); iters_out: nullable int32 [n], Newton steps
 * taken or -1 where the step failed (no convergence, singular matrix or a
 * failed temperature solve; counted by pyro_nonconverged).
 * Work arrays (about 8 (N^2 + 2N + 3) bytes per state, plus the kept FP32
 * factors with cn_newton=chord, in chunks of at most 8 GiB) are allocated on
 * first use and kept by the handle; calls on one handle must not overlap on the
 * GPU.  Returns
 * PYRO_EINVAL for dt < 0, tol <= 0 or max_newton outside [1, 1000]. */
int pyro_cn_step(const pyro_mech* mech, int64_t n, double dt, const double* rho, const double* T,
                 const double* Y, double tol, int max_newton, double* T_out, double* Y_out,
                 int32_t* iters_out, void* stream);

/* Mixture-averaged transport properties (Sec. A.2) from the mechanism's transport
 * section (PYRO_EMECH if it has none):
 *   mu_k = sqrt(T) (sum_m b_km ln^m T)^2, kappa_k = sqrt(T) sum_m c_km ln^m T,
 *   D_kj = sqrt(T) sum_m a_kjm ln^m T  (m = 0..4; fits as printed, no pressure factor);
 *   mu = sum_k X_k mu_k / sum_j Phi_kj X_j with Wilke's
 *     Phi_kj = [1 + sqrt((mu_k/mu_j) sqrt(W_j/W_k))]^2 / sqrt(8 (1 + W_k/W_j))
 *     (Eq. mixavg_viscosity);
 *   kappa = (sum_k X_k kappa_k + (sum_k X_k/kappa_k)^-1) / 2 (Eq. mixavg_conductivity);
 *   D_km = (W - X_k W_k)/W (sum_{j != k} X_j/D_kj)^-1 (Eq. diff_mix_rule);
 *   X_k = W Y_k / W_k the mole fractions.
 * T: [n] K; Y: [N][n]; mu [n] Pa s, kappa [n] W/(m K), D_mix [N][n] m^2/s out, each
 * nullable (at least one given).  D_mix of a species is undefined (0/0) where it
 * is the only species present. */
int pyro_transport(const pyro_mech* mech, int64_t n, const double* T, const double* Y, double* mu,
                   double* kappa, double* D_mix, void* stream);

/* ---- Learned initial guess for the Newton temperature solve ----------------
 * Not in the paper (its Newton starts from a fixed guess, Sec. 4.3 listing of
 * the JAX source term): a small MLP x -> 64 -> 64 -> 1 with SiLU, where the
 * D = N+1 features are x_0 = (e - e_mean)/e_std and x_{1+k} = N Y_k (Y_k
 * truncated to float first), and the output y gives
 * T_guess = clip(T_mean + T_std y, 200 K, 3500 K).  BF16
 * weights and activations (inputs, both hidden layers) with FP32 accumulation;
 * inference runs on the tensor cores inside the temperature kernel
 * (pyro_temperature with guess_mode 1), which still runs the full FP64 Newton
 * solve to the same tolerance and falls back to 1200 K where the iteration from
 * the guess fails.  Parameters (FP32 master copy, count pyro_mlp_n_params):
 *   W1[64][D], b1[64], W2[64][64], b2[64], w3[64], b3   (row-major)
 * norm4 = (e_mean, e_std, T_mean, T_std).  Supported for N <= 63 species. */
int pyro_mlp_n_params(const pyro_mech* mech);
int pyro_mlp_set_params(pyro_mech* mech, const double* params, const double* norm4);
int pyro_mlp_get_params(const pyro_mech* mech, double* params, double* norm4);

/* Train the network on device arrays T[n], Y[N][n]: the library computes e from
 * (T, Y) with its energy kernel, sets the normalisation from the data,
 * initialises the weights (seeded) and runs Adam on the mean squared error of
 * the normalised temperature with hand-written forward/backward kernels.
 * options: NULL or "epochs=1;batch=1024;lr=1e-2;seed=1" (the defaults;
 * cosine-decayed learning rate).  final_loss
 * (nullable) receives the last batch's loss.  Synchronous. */
int pyro_mlp_train(pyro_mech* mech, int64_t n, const double* T, const double* Y, const char* options,
                   double* final_loss, void* stream);

/* Loss (mean squared error of y against (T - T_mean)/T_std) and its gradient
 * over the n device states (e, Y, T), with the training kernel's arithmetic;
 * grad is a host array of pyro_mlp_n_params doubles.  Synchronous. */
int pyro_mlp_grad(const pyro_mech* mech, int64_t n, const double* e, const double* Y, const double* T,
                  double* loss, double* grad);

/* The network alone on the tensor cores: y_out[n] (normalised output) and
 * T_guess[n]. */
int pyro_mlp_guess(const pyro_mech* mech, int64_t n, const double* e, const double* Y, double* y_out,
                   double* T_guess, void* stream);

/* Save / load the parameters and normalisation (versioned binary "PYROMLP1"). */
int pyro_mlp_save(const pyro_mech* mech, const char* path);
int pyro_mlp_load(pyro_mech* mech, const char* path);

/* Net production rates for callers that cannot allocate device memory.
 * No counterpart in the paper: this is a deployment variant of
 * pyro_net_production_rates.  Some callers cannot call cudaMalloc while they
 * evaluate the chemistry -- for example a solver whose memory pool already
 * holds the whole device, or a time-step loop that must not take cudaMalloc's
 * device-wide synchronisation -- and the host-pointer path above allocates
 * staging buffers.  This entry point allocates nothing: the arrays (host or
 * device pointers, same layout and meaning as pyro_net_production_rates) and
 * the Newton failure counter are staged through one fixed scratch array of
 * PYRO_NOALLOC_SCRATCH_BYTES that the library holds as a static device
 * variable.  The array's 32 MiB are taken on a GPU when the first mechanism
 * handle is loaded there (pyro_mech_load, which may allocate), and the GPU
 * keeps them until the process exits.
 *  - Limit: the staged arrays need about 8 (2N + 3) bytes per state (N
 *    species), so one call takes at most ~32 MiB / (8 (2N + 3)) states
 *    (about 38 000 for 53 species); larger n returns PYRO_EINVAL with a message
 *    giving the limit.
 *  - pyro_mech_load also looks up the scratch's device address on its device
 *    (cudaGetSymbolAddress), so no call of this entry point does any set-up;
 *    call it only on the device the handle was loaded on.
 *  - Every call on a device shares the one scratch array, which keeps the
 *    previous call's contents (the failure counter is cleared by each call):
 *    calls that overlap on the GPU (other streams, other host threads) race.
 *  - It runs the same kernel as pyro_net_production_rates on this handle (one
 *    thread or one warp per state, see variant=).  With the thread kernel and
 *    the species arrays in the handle's global scratch (store=global, e.g. 160
 *    species) it also uses that scratch, so it must not overlap on the GPU with
 *    a pyro_net_production_rates call on the same handle either.
 *  - The call is synchronous (returns after the results are copied out) and
 *    returns PYRO_ENOCONV if a Newton solve failed (input_is_energy != 0). */
#define PYRO_NOALLOC_SCRATCH_BYTES (32u << 20)
int pyro_net_production_rates_noalloc(const pyro_mech* mech, int64_t n, const double* rho,
                                      const double* T_or_e, int input_is_energy, const double* Y,
                                      double* T_out, double* omega_out, void* stream);

/* Points whose Newton solve failed since the last call (synchronises `stream`,
 * then resets the device counter). */
int pyro_nonconverged(const pyro_mech* mech, void* stream, int64_t* count);

/* Diagnostic: the library's device exp (fn 0), log (fn 1) or reciprocal (fn 2)
 * over x[n] -> y[n], for accuracy checks against a reference libm. */
int pyro_math_eval(const pyro_mech* mech, int fn, int64_t n, const double* x, double* y,
                   void* stream);

/* Message of the calling thread's last failure ("" if none). */
const char* pyro_last_error(void);

/* Library version (major*10000 + minor*100 + patch). */
int pyro_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PYRO_H */
