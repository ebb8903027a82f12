// Molecular dynamics of the same model (Sec. II.D): velocity Verlet with a
// Nose-Hoover thermostat, on the fixed-point positions of the MC state.
#pragma once

#include <cuda_runtime.h>

#include "flipmc_types.h"

namespace flipmc {

// Device state of an MD run: velocities and forces per site (site order),
// thermostat variables per replica.
struct MdDev {
    double *v;         // 3 per site
    double *F;         // 3 per site
    double *xi;        // per replica: thermostat friction
    double *eta;       // per replica: its time integral (for the conserved energy)
    double *K;         // per replica: kinetic energy at the last thermostat step
    const double *T;   // per replica: bath temperature
    const double *Q;   // per replica: thermostat mass g T tau^2, g = 3 N
    double *scale;     // per replica: exp(-xi dt/2) of the current xi
    double *part;      // per chunk: partial kinetic energy
    const int *chunk_a0;     // per chunk: first atom (global); [n_chunks] = all atoms
    const int *rep_chunk0;   // per replica: first chunk; [n_rep] = n_chunks
    int n_chunks;
    int fp32_forces;   // 1: pair forces in FP32 (velocities, positions and thermostat stay FP64)
    double dt;
    double hdt;        // dt / 2
};

constexpr int kMdChunk = 2048;   // atoms per block of the kinetic-energy partial sums

// Thermostat half step, then the scaling and the first half kick (start of a step).
void launch_md_begin(const DevState &d, const MdDev &m, cudaStream_t st);
// Positions q += rint(v dt / h) on the records of buf (cell-sorted), periodic images counted.
void launch_md_drift(const DevState &d, int buf, const MdDev &m, cudaStream_t st);
// Forces on every atom from its partners in the 27 (or 8) neighbour cells of buf (FP64, or FP32 pair terms).
void launch_md_forces(const DevState &d, int buf, const MdDev &m, cudaStream_t st);
// Second half kick, the scaling, then the thermostat half step (end of a step).
void launch_md_end(const DevState &d, const MdDev &m, cudaStream_t st);

}  // namespace flipmc
