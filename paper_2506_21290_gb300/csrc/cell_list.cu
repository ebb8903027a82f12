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

// The same scan for large grids, in three kernels over blocks of 1024 cells
// (256 threads, 4 consecutive cells each, coalesced): the block totals, an
// exclusive scan of the totals (one block), then each block's prefixes from
// its offset.
constexpr int kScanCells = 1024;

// block-wide inclusive scan of one value per thread (256 threads); total out
__device__ __forceinline__ int scan256(int v, int *warp_tot, int &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    int before = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const int t = warp_tot[w];
        if (w < wid) before += t;
        total += t;
    }
    __syncthreads();
    return before + x;
}

__global__ void __launch_bounds__(256) cl_scan_part_kernel(DevState d)
{
    __shared__ int warp_tot[8];
    const int i0 = blockIdx.x * kScanCells + 4 * threadIdx.x;
    int v = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) v += (i0 + k < d.n_cells) ? d.cell_count[i0 + k] : 0;
    int total;
    scan256(v, warp_tot, total);
    if (threadIdx.x == 0) d.scan_part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(256) cl_scan_top_kernel(DevState d, int nb)
{
    __shared__ int warp_tot[8];
    __shared__ int carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 256) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? d.scan_part[i] : 0;
        int total;
        const int incl = scan256(v, warp_tot, total);
        const int carry = carry_s;
        if (i < nb) d.scan_part[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + total;
        __syncthreads();
    }
    if (threadIdx.x == 0) d.cell_start[d.n_cells] = carry_s;
}

__global__ void __launch_bounds__(256) cl_scan_apply_kernel(DevState d)
{
    __shared__ int warp_tot[8];
    const int i0 = blockIdx.x * kScanCells + 4 * threadIdx.x;
    int v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (i0 + k < d.n_cells) ? d.cell_count[i0 + k] : 0;
    const int sum = v[0] + v[1] + v[2] + v[3];
    int total;
    int run = d.scan_part[blockIdx.x] + scan256(sum, warp_tot, total) - sum;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (i0 + k < d.n_cells) d.cell_start[i0 + k] = run;
        run += v[k];
    }
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
    if (d.scan_part != nullptr && d.n_cells > 8 * kScanCells) {
        const int nb = (d.n_cells + kScanCells - 1) / kScanCells;
        cl_scan_part_kernel<<<nb, 256, 0, st>>>(d);
        cl_scan_top_kernel<<<1, 256, 0, st>>>(d, nb);
        cl_scan_apply_kernel<<<nb, 256, 0, st>>>(d);
    } else {
        cl_scan_kernel<<<1, 1024, 0, st>>>(d);
    }
    cl_scatter_kernel<<<nb, tb, 0, st>>>(d, buf_in, buf_out);
    const int wpb = 8;
    cl_order_kernel<<<(d.n_cells + 4 * wpb - 1) / (4 * wpb), 32 * wpb, 0, st>>>(d, buf_out);
}

}  // namespace flipmc
