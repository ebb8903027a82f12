// Cell list by counting sort (count -> exclusive scan -> scatter -> order by
// site index within each cell), as separate kernels.  One pass per sweep: an
// accepted move never takes an atom out of its cell, so the list stays valid
// for all 8 colours.  The persistent sweep kernel runs the same item bodies
// (cell_list_dev.cuh) between grid barriers.
#include "cell_list.h"
#include "cell_list_dev.cuh"

namespace flipmc {

__global__ void cl_count_kernel(DevState d, int buf)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < d.n_sites) cl_count_item(d, buf, g, d.ctr[d.rep_of_site[g]].sweep, d.cell_count);
}

// Exclusive scan of cell_count into cell_start (n_cells + 1 entries), one
// block of 1024 threads, 4 consecutive cells per thread per tile.
__global__ void __launch_bounds__(1024) cl_scan_kernel(DevState d)
{
    __shared__ int warp_tot[32];
    __shared__ int carry_s;
    const int n = d.n_cells;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 4 * 1024) {
        const int i0 = base + 4 * tid;
        int v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (i0 + k < n) ? d.cell_count[i0 + k] : 0;
        const int tsum = v[0] + v[1] + v[2] + v[3];
        int x = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int carry = carry_s;
        int run = carry + (wid > 0 ? warp_tot[wid - 1] : 0) + x - tsum;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < n) d.cell_start[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == 1023) carry_s = run;
        __syncthreads();
    }
    if (tid == 0) d.cell_start[n] = carry_s;
}

__global__ void cl_scatter_kernel(DevState d, int buf_in, int buf_out)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < d.n_sites) cl_scatter_item(d, buf_in, buf_out, g);
}

// One warp per four cells.
__global__ void cl_order_kernel(DevState d, int buf)
{
    const int lane = threadIdx.x & 31;
    const int c = 4 * (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    if (c < d.n_cells) cl_order_cells4(d, buf, c, lane);
}

void launch_cell_list(const DevState &d, int buf_in, int buf_out, cudaStream_t st)
{
    const int tb = 256;
    const int nb = (d.n_sites + tb - 1) / tb;
    cudaMemsetAsync(d.cell_count, 0, sizeof(int) * d.n_cells, st);
    cl_count_kernel<<<nb, tb, 0, st>>>(d, buf_in);
    cl_scan_kernel<<<1, 1024, 0, st>>>(d);
    cl_scatter_kernel<<<nb, tb, 0, st>>>(d, buf_in, buf_out);
    const int wpb = 8;
    cl_order_kernel<<<(d.n_cells + 4 * wpb - 1) / (4 * wpb), 32 * wpb, 0, st>>>(d, buf_out);
}

}  // namespace flipmc
