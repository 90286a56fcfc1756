// pv_terms.h -- the weights and shape constants of AutoDock Vina's pair terms (Trott & Olson 2010;
// the scoring function the paper's engine evaluates, Eq. 3), shared by the kernels and the host
// code that prepares the intra-pair records. Plain C++, no CUDA.
#pragma once

namespace pv {

constexpr float kWGauss1 = -0.0356f;
constexpr float kWGauss2 = -0.00516f;
constexpr float kWRepulsion = 0.840f;
constexpr float kWHydrophobic = -0.0351f;
constexpr float kWHBond = -0.587f;
constexpr float kWRot = 0.0585f;
constexpr float kCutoff = 8.0f;
constexpr float kCutoff2 = 64.0f;
// hydrophobic term: 1 for d < 0.5, linear to 0 at d = 1.5; H-bond term: 1 for d < -0.7, linear to
// 0 at d = 0 (d the surface distance)
constexpr float kHydGood = 0.5f, kHydBad = 1.5f;
constexpr float kHBondGood = -0.7f, kHBondBad = 0.0f;

}  // namespace pv
