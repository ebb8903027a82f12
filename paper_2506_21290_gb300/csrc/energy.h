// Energy and time-correlation kernels.
#pragma once

#include <cuda_runtime.h>

#include "flipmc_types.h"

namespace flipmc {

// Time origin of the correlation functions (Sec. III.B).
struct ObsState {
    long long *X0;   // 3 per site: unwrapped fixed point at t0
    int *kref;       // per molecule: slot of the atom that was type B at t0
    double *u0;      // 3 per molecule: unit orientation at t0
};

// FP64 energy per replica into e_out_dev[n_rep]; e_site is n_sites scratch.
void launch_energy(const DevState &d, int buf, double *e_site, double *e_out_dev, cudaStream_t st);
// unwrapped positions (3 per site) and types in site order
void launch_gather(const DevState &d, int buf, long long *X, int *types, cudaStream_t st);
void launch_set_t0(const DevState &d, const long long *X, const int *types, const ObsState &o, cudaStream_t st);
// out[3 r + {0,1,2}] = F_s, F_s^cm, C_2 of replica r
void launch_observables(const DevState &d, const long long *X, const ObsState &o, const double *qa, int nqa,
                        const double *qc, int nqc, double *fs_site, double *fscm_mol, double *c2_mol, double *out,
                        cudaStream_t st);

}  // namespace flipmc
