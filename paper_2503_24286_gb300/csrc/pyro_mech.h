// Mechanism description used by the emitter and the runtime (host side).
//
// A mechanism is the data of the paper's formulation (Sec. A.1): species with
// molecular weights and two-range NASA-7 coefficients (Eq. nasa_poly,
// Eq. nasa_poly_c), and reactions (Eq. reactions) with mass-action rates of
// progress (Eq. reaction_rates), Arrhenius coefficients (Eq. rate_coeff),
// optional third-body efficiencies and Troe falloff parameters.
#pragma once

#include <string>
#include <utility>
#include <vector>

namespace pyro {

struct Species {
  std::string name;
  std::vector<std::pair<int, int>> composition;   // (element index, atom count)
  double W = 0.0;                                 // molecular weight, kg/kmol
  double t_low = 0.0, t_mid = 0.0, t_high = 0.0;  // NASA-7 ranges, K
  double low[7] = {0}, high[7] = {0};             // a1..a7 below / above t_mid
};

enum ReactionKind { RX_ARRHENIUS = 0, RX_THREEBODY = 1, RX_FALLOFF = 2, RX_PLOG = 3 };

// PLOG node: rate coefficient A T^b exp(-theta/T) at pressure p (Pa)
struct PlogNode { double p = 0.0, A = 0.0, b = 0.0, theta = 0.0; };

struct Reaction {
  ReactionKind kind = RX_ARRHENIUS;
  bool reversible = true;
  bool duplicate = false;
  std::vector<std::pair<int, int>> reactants;     // (species, stoichiometric coefficient nu')
  std::vector<std::pair<int, int>> products;      // (species, nu'')
  double A = 0.0, b = 0.0, theta = 0.0;           // k = A T^b exp(-theta/T)  (high-pressure limit for falloff)
  std::vector<std::pair<int, double>> efficiencies;   // third-body efficiencies (default 1)
  bool has_low = false;
  double A0 = 0.0, b0 = 0.0, theta0 = 0.0;        // low-pressure limit k0
  int n_troe = 0;                                 // 0: Lindemann, 3 or 4: Troe (a, T3, T1[, T2])
  double troe[4] = {0, 0, 0, 0};
  int n_sri = 0;                                  // 0, or 3 / 5: SRI falloff (a, b, c[, d, e]), d = 1, e = 0 by default
  double sri[5] = {0, 0, 0, 1, 0};
  std::vector<PlogNode> plog;                     // RX_PLOG: nodes in increasing pressure
};

// Mixture-averaged transport data (Sec. A.2): per-species fits of viscosity
// mu_k = sqrt(T) (sum_m b_km ln^m T)^2 and conductivity kappa_k = sqrt(T) sum_m c_km ln^m T,
// and symmetric binary-diffusivity fits D_kj = sqrt(T) sum_m a_kjm ln^m T, m = 0..4.
struct TransportFits {
  std::vector<double> visc, cond;   // [N][5]
  std::vector<double> diff;         // [N][N][5], symmetric, diagonal unused
};

struct Mechanism {
  std::string name;
  std::vector<std::string> element_names;
  std::vector<double> element_weights;
  std::vector<Species> species;
  std::vector<Reaction> reactions;
  bool has_transport = false;
  TransportFits transport;
  int n_species() const { return (int)species.size(); }
  int n_reactions() const { return (int)reactions.size(); }
};

// Parse the text interchange format ("pyro-mech 1").  Returns false and sets err.
bool parse_mechanism_file(const std::string& path, Mechanism& m, std::string& err);

// Structural and physical checks: indices, integer element balance of every
// reaction, positive pre-exponential factors, NASA ranges, cp/R > 1 (so that
// c_v > 0 and e(T) is invertible) sampled over [t_low, t_high], Troe data
// consistency.  Returns false and sets err.
bool validate_mechanism(const Mechanism& m, std::string& err);

}  // namespace pyro
