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

// FP64 energy per replica into e_out_dev[n_rep]; e_cell is n_cells scratch.
void launch_energy(const DevState &d, int buf, double *e_cell, double *e_out_dev, cudaStream_t st);
// Periodic drift check: drift[2r] = |e_run - E| / |E| (last), drift[2r+1] its
// largest value; one recompute counted; e_run restarts from E[r].
void launch_drift(const DevState &d, const double *E, double *drift, cudaStream_t st);
// S(q) per (replica, wavevector): out[r * n_q + k] = |sum_i exp(i q_k . x_i)|^2 / N.
void launch_sq(const DevState &d, const long long *X, const double *qv, int n_q, double *out, cudaStream_t st);
// Pair-distance counts per replica and bin (every pair once); counts zeroed by the caller.
void launch_pair_hist(const DevState &d, const long long *X, int max_sites, double dr, int n_bins,
                      unsigned long long *counts, cudaStream_t st);
// FP64 pair virial sum W = sum_{i<j} -r dphi/dr per replica into w_out_dev[n_rep].
void launch_virial(const DevState &d, int buf, double *w_cell, double *w_out_dev, cudaStream_t st);
// unwrapped positions (3 per site) and types in site order
void launch_gather(const DevState &d, int buf, long long *X, int *types, cudaStream_t st);
void launch_set_t0(const DevState &d, const long long *X, const int *types, const ObsState &o, cudaStream_t st);
// out[3 r + {0,1,2}] = F_s, F_s^cm, C_2 of replica r
void launch_observables(const DevState &d, const long long *X, const ObsState &o, const double *qa, int nqa,
                        const double *qc, int nqc, double *fs_site, double *fscm_mol, double *c2_mol, double *out,
                        cudaStream_t st);

// Multiple-origin correlations: the origins live in slots; each slot holds an
// ObsState's arrays (slot s at X0 + 3 N s, kref + M s, u0 + 3 M s).
struct CorrDev {
    const long long *X0;
    const int *kref;
    const double *u0;
    size_t n_sites;             // all replicas
    const double *qa;           // n_qa wavevectors (atoms), 3 each
    const double *qc;           // n_qc wavevectors (centres of mass)
    int n_qa, n_qc;
    const int *chunk_m0;        // per chunk: first molecule (global index), chunk_m0[n_chunks] = total molecules
    int n_chunks;
    const int *rep_chunk0;      // per replica: first chunk; [n_rep] = n_chunks
    double *partials;           // CORR_PART per (pair, chunk)
    double *acc;                // MC_CORR_NSUM per (replica, lag)
    int n_lags;
};

constexpr int kCorrMaxPairs = 32;       // (origin, lag) pairs per launch
constexpr int kCorrChunk = 256;         // molecules per block of the per-particle pass (one per thread)
constexpr int kCorrPart = 8;            // partial sums per (pair, chunk)

// The (origin slot, lag index) pairs measured at one time.
struct CorrPairs {
    int n;
    int slot[kCorrMaxPairs];
    int lag[kCorrMaxPairs];
};

// Per-particle correlations of each pair against the current unwrapped
// positions X, summed per replica into the accumulators (fixed order).
void launch_corr_sample(const DevState &d, const long long *X, const CorrDev &c, const CorrPairs &p, cudaStream_t st);

}  // namespace flipmc
