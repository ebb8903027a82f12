// Cell list build (counting sort) and the sweep's launch sequence.
#pragma once

#include <cuda_runtime.h>

#include "flipmc_types.h"

namespace flipmc {

__global__ void cl_count_kernel(DevState d, int buf);
__global__ void cl_scan_kernel(DevState d);
__global__ void cl_scatter_kernel(DevState d, int buf_in, int buf_out);
__global__ void cl_order_kernel(DevState d, int buf);

// count + scan + scatter + per-cell ordering: records of buf_in, cell-sorted into buf_out.
void launch_cell_list(const DevState &d, int buf_in, int buf_out, cudaStream_t st);

// Attempt-log destination of a logged sweep (null base: no log).
struct LogArgs {
    mc_log_entry *base;
    int n_sweeps;         // sweeps recorded by this call
    uint64_t sweep0;      // first sweep number recorded
};

// the 8 colour phases of one sweep on buf, then the per-sweep finalisation
void launch_phases(const DevState &d, int buf, int warps_per_block, const LogArgs &lg, cudaStream_t st);
// the same two stages, separately (for per-stage timing)
void launch_colour_phases(const DevState &d, int buf, int warps_per_block, const LogArgs &lg, cudaStream_t st);
void launch_finalize(const DevState &d, cudaStream_t st);
size_t phase_smem_bytes(int stencil_cap, int warps_per_cell);
int phase_set_smem_limit(int bytes_needed);

// Persistent sweeps: co-resident blocks for one cooperative launch (0 when the
// device cannot launch cooperatively), and the launch itself (n_sweeps whole
// sweeps starting from records in buf; bar: 2 zeroed words; scan_tot: one int
// per block).  Returns 0 or a cudaError_t.
int persistent_grid(const DevState &d, int warps_per_cell, int max_blocks);
int launch_persistent(const DevState &d, int buf, int n_sweeps, int warps_per_cell, int grid, unsigned int *bar,
                      int *scan_tot, cudaStream_t st);

// compute capability the sweep kernels were built for (cudaFuncAttributes
// binaryVersion, e.g. 103), or -1
int sweep_binary_version();

// the calling thread's last error, as mc_last_error() reports it; returns code
int record_error(int code, const char *msg);

}  // namespace flipmc
