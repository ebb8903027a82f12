// Cell list by counting sort (count -> exclusive scan -> scatter -> order by
// site index within each cell).  One pass per sweep: an accepted move never
// takes an atom out of its cell, so the list stays valid for all 8 colours.
//
// The grid of a replica is n_c^3 cells of side L/n_c, shifted by the sweep's
// random 32-bit offset (x + shift) per axis; an atom's cell along an axis is
// ((q + shift) * n_c) >> 32 on its 32-bit fixed-point coordinate q.
#include "cell_list.h"
#include "flipmc_device.cuh"

namespace flipmc {

// Cell of every atom under the sweep's shift; slot by atomic count.
// Also publishes the replica's shift (written by the replica's first atom).
__global__ void cl_count_kernel(DevState d, int buf)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= d.n_sites) return;
    const int r = d.rep_of_site[g];
    const RepInfo ri = d.rep[r];
    RepCtr *ct = d.ctr + r;
    const U4 s = rng_block(0xFFFFFFFFu, 0xFFFFFFFFu, ct->sweep, d.par[r].seed);
    if (g == ri.site_off) {
        ct->shift[0] = s.x;
        ct->shift[1] = s.y;
        ct->shift[2] = s.z;
    }
    const uint32_t shift[3] = {s.x, s.y, s.z};
    const int4 rc = d.rec[buf][g];
    const int c = ri.cell_off + cell_local((uint32_t)rc.x, (uint32_t)rc.y, (uint32_t)rc.z, shift, ri.nc);
    d.cell_of[g] = c;
    d.slot_of[g] = atomicAdd(d.cell_count + c, 1);
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
    if (g >= d.n_sites) return;
    d.rec[buf_out][d.cell_start[d.cell_of[g]] + d.slot_of[g]] = d.rec[buf_in][g];
}

// Order the atoms of each cell by site index (the record word orders by
// molecule, then slot), so the layout after a build does not depend on the
// order in which the atomic counts were taken.  One warp per cell.
__global__ void cl_order_kernel(DevState d, int buf)
{
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= d.n_cells) return;
    const int start = d.cell_start[c];
    const int n = d.cell_start[c + 1] - start;
    int4 *seg = d.rec[buf] + start;
    if (n <= 1) return;
    if (n <= 32) {
        int4 mine = lane < n ? seg[lane] : make_int4(0, 0, 0, 0x7fffffff);
        const unsigned key = (unsigned)mine.w;
        int rank = 0;
        for (int m = 0; m < n; ++m) {
            const unsigned other = __shfl_sync(0xffffffffu, key, m);
            rank += other < key;
        }
        __syncwarp();
        if (lane < n) seg[rank] = mine;
        return;
    }
    // larger cells (small boxes only): insertion sort by one lane
    if (lane == 0) {
        for (int i = 1; i < n; ++i) {
            const int4 v = seg[i];
            int j = i - 1;
            while (j >= 0 && (unsigned)seg[j].w > (unsigned)v.w) {
                seg[j + 1] = seg[j];
                --j;
            }
            seg[j + 1] = v;
        }
    }
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
    cl_order_kernel<<<(d.n_cells + wpb - 1) / wpb, 32 * wpb, 0, st>>>(d, buf_out);
}

}  // namespace flipmc
