// Per-item bodies of the cell-list build, shared by the stand-alone kernels
// (cell_list.cu) and the persistent sweep kernel (sweep.cu).
//
// The grid of a replica is n_c^3 cells of side L/n_c, shifted by the sweep's
// random 32-bit offset per axis; an atom's cell along an axis is
// ((q + shift) * n_c) >> 32 on its 32-bit fixed-point coordinate q.
#pragma once

#include "flipmc_device.cuh"

namespace flipmc {

// Cell of atom g under the shift of sweep `sweep`; slot by atomic count in
// `counts`.  The replica's first atom also publishes the shift.
__device__ __forceinline__ void cl_count_item(const DevState &d, int buf, int g, uint64_t sweep, int *counts)
{
    const int r = d.rep_of_site[g];
    const RepInfo ri = d.rep[r];
    RepCtr *ct = d.ctr + r;
    const U4 s = rng_block(0xFFFFFFFFu, 0xFFFFFFFFu, sweep, d.par[r].seed);
    if (g == ri.site_off) {
        ct->shift[0] = s.x;
        ct->shift[1] = s.y;
        ct->shift[2] = s.z;
    }
    const uint32_t shift[3] = {s.x, s.y, s.z};
    const int4 rc = d.rec[buf][g];
    const int c = ri.cell_off + cell_local((uint32_t)rc.x, (uint32_t)rc.y, (uint32_t)rc.z, shift, ri.nc);
    d.cell_of[g] = c;
    d.slot_of[g] = atomicAdd(counts + c, 1);
}


// The random draws and the Metropolis threshold of every attempt of the sweep.
// Attempt a of cell c (a < occupancy n) is slot start(c) + a; its words are
// the Philox blocks (2a, c, sweep) and (2a+1, c, sweep) under the replica's
// seed, w0..w7.  Everything that does not depend on the state is decoded here,
// off the serial attempt chain:
//   quad 0: x = site rank (w0 n) >> 32 | move type (integer thresholds on w1)
//           << 16 | flip axis (w7 3) >> 32 << 18;
//           y, z, w = the displacement drawn from w4, w5, w6 (atom step for a
//           translation, molecule step for a molecule translation), or w4, w5,
//           w6 themselves for a rotation;
//   quad 1: x, y = w2, w3 (u = (2 u52 + 1) 2^-53 of the threshold), z, w = 0;
// and the threshold -T ln u (FP64 series in FP64 mode, __logf in FP32 mode).
__device__ __forceinline__ void attempt_randoms(const DevState &d, int r, int cellL, int slot, int a, int n)
{
    const uint64_t sweep = d.ctr[r].sweep;
    const RepParam par = d.par[r];
    const U4 b0 = rng_block((uint32_t)(2 * a), (uint32_t)cellL, sweep, par.seed);
    const U4 b1 = rng_block((uint32_t)(2 * a + 1), (uint32_t)cellL, sweep, par.seed);
    const MixDev mx = *d.mix;
    const int k = (int)(((unsigned long long)b0.x * (unsigned long long)n) >> 32);
    const int mvt = move_type(b0.y, mx);
    const int axis = (int)(((unsigned long long)b1.w * 3ull) >> 32);
    uint4 q0;
    q0.x = (uint32_t)k | ((uint32_t)mvt << 16) | ((uint32_t)axis << 18);
    if (mvt == MC_MOVE_MOL_ROT) {
        q0.y = b1.x;
        q0.z = b1.y;
        q0.w = b1.z;
    } else {
        const int32_t D = mvt == MC_MOVE_MOL_TRANS ? par.D_mol : par.D_atom;
        q0.y = (uint32_t)uniform_disp(b1.x, D);
        q0.z = (uint32_t)uniform_disp(b1.y, D);
        q0.w = (uint32_t)uniform_disp(b1.z, D);
    }
    d.att_rnd[2 * (size_t)slot] = q0;
    d.att_rnd[2 * (size_t)slot + 1] = make_uint4(b0.z, b0.w, 0u, 0u);
    const unsigned long long u52 = ((unsigned long long)b0.z << 20) | (unsigned long long)(b0.w >> 12);
    const double T = par.T;
    if (d.precision == MC_PREC_FP64) {
        const double u = __dmul_rn((double)(2ull * u52 + 1ull), 0x1p-53);
        d.att_thr64[slot] = -__dmul_rn(T, ln_series(u));
    } else {
        const float uf = __ull2float_rn(2ull * u52 + 1ull) * 0x1p-53f;
        d.att_thr32[slot] = -(float)T * __logf(uf);
    }
}

// Scatter atom g into its cell's segment at its counting slot a, and draw the
// random numbers of attempt a of that cell (when the sweep needs them): the
// cell's atoms and its attempts are both numbered 0..n-1, so one thread per
// atom covers every attempt, and the draws depend on (seed, sweep, cell, a,
// n) only, not on which atom took slot a.
__device__ __forceinline__ void cl_scatter_item(const DevState &d, int buf_in, int buf_out, int g)
{
    const int c = d.cell_of[g];
    const int start = d.cell_start[c];
    const int a = d.slot_of[g];
    d.rec[buf_out][start + a] = d.rec[buf_in][g];
    if (d.att_rnd != nullptr) {
        const int r = d.rep_of_site[g];
        attempt_randoms(d, r, c - d.rep[r].cell_off, start + a, a, d.cell_start[c + 1] - start);
    }
}

// Order the atoms of cell c by site index (the record word orders by
// molecule, then slot), so the layout after a build does not depend on the
// order in which the atomic counts were taken.  One warp.
__device__ __forceinline__ void cl_order_cell(const DevState &d, int buf, int c, int lane)
{
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
        __syncwarp();
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
    __syncwarp();
}

// Order the four cells c0 .. c0 + 3 at once, eight lanes each, when they hold
// at most eight atoms (the usual case at the paper's density); a larger cell
// is then ordered by the whole warp.  One warp.
__device__ __forceinline__ void cl_order_cells4(const DevState &d, int buf, int c0, int lane)
{
    const int sub = lane & 7, c = c0 + (lane >> 3);
    int start = 0, n = 0;
    if (c < d.n_cells) {
        start = d.cell_start[c];
        n = d.cell_start[c + 1] - start;
    }
    int4 *seg = d.rec[buf] + start;
    const bool mine_ok = sub < n && n <= 8;
    const int4 mine = mine_ok ? seg[sub] : make_int4(0, 0, 0, 0x7fffffff);
    const unsigned key = (unsigned)mine.w;
    int rank = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m) rank += __shfl_sync(0xffffffffu, key, m, 8) < key;
    __syncwarp();
    if (mine_ok && n > 1) seg[rank] = mine;
    __syncwarp();
    unsigned big = __ballot_sync(0xffffffffu, sub == 0 && n > 8);
    while (big) {
        const int k = __ffs(big) - 1;
        big &= big - 1;
        cl_order_cell(d, buf, c0 + (k >> 3), lane);
    }
}

}  // namespace flipmc
