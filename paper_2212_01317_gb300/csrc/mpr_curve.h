// Launchers of mpr_curve.cu: the unconditional e(T) curve of a data-free
// lattice and the calibration steps that read it.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_internal.h"

namespace mpr {

// Side of the data-free lattice the curve is measured on.
constexpr int kCurveSide = 64;
// Most points a curve may have.
constexpr int kCurveMaxPoints = 64;

// e_out[k] = mean E / N_bonds over n_meas sweeps after n_eq, at T[k] (device
// arrays of n_T entries).
void launch_energy_curve(const float* T, int n_T, int n_eq, int n_meas, const Model& m,
                         uint64_t seed, double* e_out, cudaStream_t s);
// Warm first iteration: two points into T0a / T0b, more into Tk[p * nblk + b].
void launch_warm_points(int nblk, int points, const int32_t* Nsp, const double* es,
                        const float* cT, const double* ce, int cn, double w, float* T0a,
                        float* T0b, float* Tk, Control* ctl, cudaStream_t s);
// T_b = T0_b (targeted blocks), 0 otherwise.
void launch_curve_T(int nblk, const int32_t* Nsp, const double* es, const float* cT,
                    const double* ce, int cn, float* T, cudaStream_t s);

}  // namespace mpr
