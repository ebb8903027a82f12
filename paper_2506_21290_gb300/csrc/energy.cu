// Total energy (Eq. 1 + Eq. 2, FP64) over the cell neighbourhoods, and the
// time correlations of Sec. III.B (Eq. 5-7).
#include "cell_list.h"
#include "energy.h"
#include "flipmc_device.cuh"

namespace flipmc {

// Energy (VIRIAL = false) or pair virial (VIRIAL = true), one warp per cell:
// every pair (i, j) with i an atom of the cell and j an atom of the 27 (or,
// for n_c = 2, the 8) neighbour cells with a larger site index.  Lane k walks
// neighbour cell k; pairs of different molecules beyond every cutoff (FP32
// screen with a 1% margin) add exactly 0 and are dropped; the others are
// gathered in order into a ring and evaluated in FP64 32 at a time, one per
// lane, so the FP64 pipe works on full warps.  Each lane sums its pairs in
// gathering order and a fixed butterfly adds the lanes: the cell's sum is the
// same on every run for a given state.
constexpr int kCellWarps = 8;       // cells per block
constexpr int kRing = 64;           // gathered pairs per warp (at most 63 waiting)

template <bool VIRIAL>
__global__ void __launch_bounds__(32 * kCellWarps) pair_cells_kernel(DevState d, int buf, double *e_cell)
{
    __shared__ int2 ring_all[kCellWarps][kRing];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int c = blockIdx.x * kCellWarps + wib;
    if (c >= d.n_cells) return;   // the whole warp
    int2 *ring = ring_all[wib];
    const int s0 = d.cell_start[c];
    const int n = d.cell_start[c + 1] - s0;
    double acc = 0.0;
    if (n > 0) {
        const int r = d.rep_of_site[s0];
        const RepInfo ri = d.rep[r];
        const ModelDev &md = *d.model;
        const int4 *rec = d.rec[buf];
        const int nc = ri.nc, cl = c - ri.cell_off;
        const int cx = cl % nc, cy = (cl / nc) % nc, cz = cl / (nc * nc);
        const bool small = nc == 2;
        const int ns = small ? 8 : 27;
        int cst = 0, cnt = 0;
        if (lane < ns) {
            int ox, oy, oz;
            if (small) {
                ox = lane & 1; oy = (lane >> 1) & 1; oz = lane >> 2;
            } else {
                ox = lane % 3 - 1; oy = (lane / 3) % 3 - 1; oz = lane / 9 - 1;
            }
            const int nb = ri.cell_off + (((cz + oz + nc) % nc) * nc + (cy + oy + nc) % nc) * nc + (cx + ox + nc) % nc;
            cst = d.cell_start[nb];
            cnt = d.cell_start[nb + 1] - cst;
        }
        const int maxc = __reduce_max_sync(0xffffffffu, cnt);
        float rc2max = 0.f;
        for (int k = 0; k < 9; ++k) rc2max = fmaxf(rc2max, md.rc2f[k]);
        const float pre = rc2max * 1.01f;
        const unsigned lt = (1u << lane) - 1u;
        int head = 0, tail = 0;   // warp-uniform
        auto eval = [&](int e) {
            const int2 p = ring[e & (kRing - 1)];
            const int4 me = rec[s0 + p.x], o = rec[p.y];
            const int dx = (int)((uint32_t)o.x - (uint32_t)me.x);
            const int dy = (int)((uint32_t)o.y - (uint32_t)me.y);
            const int dz = (int)((uint32_t)o.z - (uint32_t)me.z);
            const double r2 = r2_fixed64(dx, dy, dz, ri.h);
            const bool bonded = rec_mol(o.w) == rec_mol(me.w);
            const int ab = 3 * rec_type(me.w) + rec_type(o.w);
            acc = __dadd_rn(acc, VIRIAL ? virial64(md, r2, ab, bonded) : phi64(md, r2, ab, bonded));
        };
        for (int i = 0; i < n; ++i) {
            const int4 me = rec[s0 + i];
            const int si = rec_site(me.w), mi = rec_mol(me.w);
            for (int k = 0; k < maxc; ++k) {
                bool hit = false;
                if (k < cnt) {
                    const int4 o = rec[cst + k];
                    if (rec_site(o.w) > si) {
                        if (rec_mol(o.w) == mi) {
                            hit = true;
                        } else {
                            const float fx = (float)(int)((uint32_t)o.x - (uint32_t)me.x) * ri.hf;
                            const float fy = (float)(int)((uint32_t)o.y - (uint32_t)me.y) * ri.hf;
                            const float fz = (float)(int)((uint32_t)o.z - (uint32_t)me.z) * ri.hf;
                            hit = fx * fx + fy * fy + fz * fz <= pre;
                        }
                    }
                }
                const unsigned b = __ballot_sync(0xffffffffu, hit);
                if (hit) ring[(tail + __popc(b & lt)) & (kRing - 1)] = make_int2(i, cst + k);
                tail += __popc(b);
                if (tail - head >= 32) {
                    __syncwarp();
                    eval(head + lane);
                    head += 32;
                    __syncwarp();
                }
            }
        }
        __syncwarp();
        if (lane < tail - head) eval(head + lane);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if (lane == 0) e_cell[c] = acc;
}

// Fixed-order sum of the per-cell values of each replica (one block each).
__global__ void __launch_bounds__(256) replica_cells_sum_kernel(DevState d, const double *v, double *out)
{
    const int r = blockIdx.x;
    const RepInfo ri = d.rep[r];
    const int n = ri.nc * ri.nc * ri.nc;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s = __dadd_rn(s, v[ri.cell_off + i]);
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r] = red[0];
}

// Fixed-order sum of a per-site (or per-molecule) array over each replica.
__global__ void __launch_bounds__(256) replica_sum_kernel(DevState d, const double *v, int per_mol, double scale_inv_n,
                                                          double *out, int stride, int offset)
{
    const int r = blockIdx.x;
    const RepInfo ri = d.rep[r];
    const int n = per_mol ? ri.n_sites / 3 : ri.n_sites;
    const int off = per_mol ? ri.site_off / 3 : ri.site_off;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s = __dadd_rn(s, v[off + i]);
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)r * stride + offset] = scale_inv_n != 0.0 ? red[0] / (double)n : red[0];
}

void launch_energy(const DevState &d, int buf, double *e_cell, double *e_out_dev, cudaStream_t st)
{
    pair_cells_kernel<false><<<(d.n_cells + kCellWarps - 1) / kCellWarps, 32 * kCellWarps, 0, st>>>(d, buf, e_cell);
    replica_cells_sum_kernel<<<d.n_rep, 256, 0, st>>>(d, e_cell, e_out_dev);
}

// Drift check of the running total against a fresh FP64 recompute E, per
// replica (one thread each): the relative drift |e_run - E| / |E| into
// drift[2r] (last) and drift[2r + 1] (largest so far), one more recompute
// counted, and e_run restarted from E.
__global__ void drift_kernel(DevState d, const double *E, double *drift)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.n_rep) return;
    const double e = E[r];
    const double rel = fabs(d.e_run[r] - e) / fabs(e);
    drift[2 * r] = rel;
    drift[2 * r + 1] = fmax(drift[2 * r + 1], rel);
    d.stats[(size_t)r * STAT_N + STAT_RECOMP] += 1;
    d.e_run[r] = e;
}

void launch_drift(const DevState &d, const double *E, double *drift, cudaStream_t st)
{
    drift_kernel<<<(d.n_rep + 127) / 128, 128, 0, st>>>(d, E, drift);
}

void launch_virial(const DevState &d, int buf, double *w_cell, double *w_out_dev, cudaStream_t st)
{
    pair_cells_kernel<true><<<(d.n_cells + kCellWarps - 1) / kCellWarps, 32 * kCellWarps, 0, st>>>(d, buf, w_cell);
    replica_cells_sum_kernel<<<d.n_rep, 256, 0, st>>>(d, w_cell, w_out_dev);
}

// Unwrapped fixed-point positions and types in site-index order.
__global__ void gather_kernel(DevState d, int buf, long long *X, int *types)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= d.n_sites) return;
    const int r = d.rep_of_site[g];
    const int off = d.rep[r].site_off;
    const int4 rc = d.rec[buf][g];
    const int s = off + rec_site(rc.w);
    X[3 * s + 0] = (long long)(uint32_t)rc.x + ((long long)d.img[3 * s + 0] << 32);
    X[3 * s + 1] = (long long)(uint32_t)rc.y + ((long long)d.img[3 * s + 1] << 32);
    X[3 * s + 2] = (long long)(uint32_t)rc.z + ((long long)d.img[3 * s + 2] << 32);
    types[s] = rec_type(rc.w);
}

// Orientation of molecule m (global index): centroid -> site kref, from the
// wrapped positions with intramolecular minimum images (equal masses).
__device__ void orientation(const long long *X, int m, int kref, double h, double *u)
{
    const long long *x0 = X + 9 * (size_t)m;
    double rel[3][3];
    for (int k = 0; k < 3; ++k)
        for (int ax = 0; ax < 3; ++ax) rel[k][ax] = (double)(int)((uint32_t)x0[3 * k + ax] - (uint32_t)x0[ax]) * h;
    double n2 = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        const double cm = ((rel[0][ax] + rel[1][ax]) + rel[2][ax]) / 3.0;
        u[ax] = rel[kref][ax] - cm;
        n2 += u[ax] * u[ax];
    }
    const double inv = 1.0 / sqrt(n2);
    for (int ax = 0; ax < 3; ++ax) u[ax] *= inv;
}

__global__ void set_t0_kernel(DevState d, const long long *X, const int *types, ObsState o)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= d.n_sites / 3) return;
    for (int k = 0; k < 9; ++k) o.X0[9 * (size_t)m + k] = X[9 * (size_t)m + k];
    int kref = 0;
    for (int s = 2; s >= 0; --s)
        if (types[3 * m + s] == 1) kref = s;
    o.kref[m] = kref;
    const int r = d.rep_of_site[3 * m];
    double u[3];
    orientation(X, m, kref, d.rep[r].h, u);
    for (int ax = 0; ax < 3; ++ax) o.u0[3 * (size_t)m + ax] = u[ax];
}

// Per molecule: F_s of its three atoms, F_s^cm and C_2 (Eq. 5-7).
__global__ void observables_kernel(DevState d, const long long *X, ObsState o, const double *qa, int nqa,
                                   const double *qc, int nqc, double *fs_site, double *fscm_mol, double *c2_mol)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= d.n_sites / 3) return;
    const int r = d.rep_of_site[3 * m];
    const double h = d.rep[r].h;
    double dx[3][3];
    for (int k = 0; k < 3; ++k)
        for (int ax = 0; ax < 3; ++ax)
            dx[k][ax] = (double)(X[9 * (size_t)m + 3 * k + ax] - o.X0[9 * (size_t)m + 3 * k + ax]) * h;
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int q = 0; q < nqa; ++q)
            s += cos(qa[3 * q] * dx[k][0] + qa[3 * q + 1] * dx[k][1] + qa[3 * q + 2] * dx[k][2]);
        fs_site[3 * (size_t)m + k] = s / (double)nqa;
    }
    double cm[3];
    for (int ax = 0; ax < 3; ++ax) cm[ax] = ((dx[0][ax] + dx[1][ax]) + dx[2][ax]) / 3.0;
    double s = 0.0;
    for (int q = 0; q < nqc; ++q) s += cos(qc[3 * q] * cm[0] + qc[3 * q + 1] * cm[1] + qc[3 * q + 2] * cm[2]);
    fscm_mol[m] = s / (double)nqc;
    double u[3];
    orientation(X, m, o.kref[m], h, u);
    const double x = u[0] * o.u0[3 * (size_t)m] + u[1] * o.u0[3 * (size_t)m + 1] + u[2] * o.u0[3 * (size_t)m + 2];
    c2_mol[m] = 1.5 * x * x - 0.5;
}

// The per-molecule quantities of one (origin, time) pair that the sums need:
// F_s of the three atoms (their sum and sum of squares), F_s^cm, C_2, and the
// products of Eq. chi4 and of the Pearson coefficient.
struct CorrVals {
    double v[7];   // sum_k fs_k, sum_k fs_k^2, fcm, fcm^2, c2, c2^2, c2 fcm
};

__device__ CorrVals corr_molecule(const long long *X, const long long *X0, int kref, const double *u0, int m, double h,
                                  const double *qa, int nqa, const double *qc, int nqc)
{
    double dx[3][3];
    for (int k = 0; k < 3; ++k)
        for (int ax = 0; ax < 3; ++ax) dx[k][ax] = (double)(X[9 * (size_t)m + 3 * k + ax] - X0[9 * (size_t)m + 3 * k + ax]) * h;
    CorrVals o;
    o.v[0] = 0.0;
    o.v[1] = 0.0;
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int q = 0; q < nqa; ++q)
            s += cos(qa[3 * q] * dx[k][0] + qa[3 * q + 1] * dx[k][1] + qa[3 * q + 2] * dx[k][2]);
        const double f = s / (double)nqa;
        o.v[0] += f;
        o.v[1] += f * f;
    }
    double cm[3];
    for (int ax = 0; ax < 3; ++ax) cm[ax] = ((dx[0][ax] + dx[1][ax]) + dx[2][ax]) / 3.0;
    double s = 0.0;
    for (int q = 0; q < nqc; ++q) s += cos(qc[3 * q] * cm[0] + qc[3 * q + 1] * cm[1] + qc[3 * q + 2] * cm[2]);
    const double fcm = s / (double)nqc;
    double u[3];
    orientation(X, m, kref, h, u);
    const double x = u[0] * u0[0] + u[1] * u0[1] + u[2] * u0[2];
    const double c2 = 1.5 * x * x - 0.5;
    o.v[2] = fcm;
    o.v[3] = fcm * fcm;
    o.v[4] = c2;
    o.v[5] = c2 * c2;
    o.v[6] = c2 * fcm;
    return o;
}

// Block (chunk, pair): the chunk's molecules (one replica's), each thread in
// ascending order, then a fixed tree over the block's threads.
__global__ void __launch_bounds__(256) corr_chunk_kernel(DevState d, const long long *X, CorrDev c, CorrPairs p)
{
    const int chunk = blockIdx.x, pr = blockIdx.y;
    const int m0 = c.chunk_m0[chunk], m1 = c.chunk_m0[chunk + 1];
    const int slot = p.slot[pr];
    const size_t M = c.n_sites / 3;
    const long long *X0 = c.X0 + (size_t)slot * 3 * c.n_sites;
    const int *kref = c.kref + (size_t)slot * M;
    const double *u0 = c.u0 + (size_t)slot * 3 * M;
    const double h = d.rep[d.rep_of_site[3 * m0]].h;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int m = m0 + threadIdx.x; m < m1; m += 256) {
        const CorrVals v = corr_molecule(X, X0, kref[m], u0 + 3 * (size_t)m, m, h, c.qa, c.n_qa, c.qc, c.n_qc);
        for (int j = 0; j < 7; ++j) acc[j] = __dadd_rn(acc[j], v.v[j]);
    }
    __shared__ double red[7][256];
    for (int j = 0; j < 7; ++j) red[j][threadIdx.x] = acc[j];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int j = 0; j < 7; ++j) red[j][threadIdx.x] = __dadd_rn(red[j][threadIdx.x], red[j][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x < 7) c.partials[((size_t)pr * c.n_chunks + chunk) * kCorrPart + threadIdx.x] = red[threadIdx.x][0];
}

// Block (pair, replica): the replica's chunk sums (thread k takes chunks k,
// k + 128, ... in order, then a fixed tree over the threads), then the
// sample's contribution to the replica's accumulators of the pair's lag.
// Different origins never share a lag at one time, so each accumulator has
// one writer per launch.
__global__ void __launch_bounds__(128) corr_finish_kernel(DevState d, CorrDev c, CorrPairs p)
{
    const int pr = blockIdx.x / d.n_rep, r = blockIdx.x - pr * d.n_rep;
    double S[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int k = c.rep_chunk0[r] + threadIdx.x; k < c.rep_chunk0[r + 1]; k += 128)
        for (int j = 0; j < 7; ++j) S[j] = __dadd_rn(S[j], c.partials[((size_t)pr * c.n_chunks + k) * kCorrPart + j]);
    __shared__ double red[7][128];
    for (int j = 0; j < 7; ++j) red[j][threadIdx.x] = S[j];
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int j = 0; j < 7; ++j) red[j][threadIdx.x] = __dadd_rn(red[j][threadIdx.x], red[j][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    for (int j = 0; j < 7; ++j) S[j] = red[j][0];
    const double M = (double)(d.rep[r].n_sites / 3), N = 3.0 * M;
    const double fs = S[0] / N, fcm = S[2] / M, c2 = S[4] / M;
    double *a = c.acc + ((size_t)r * c.n_lags + p.lag[pr]) * MC_CORR_NSUM;
    a[0] += 1.0;
    a[1] += fs;
    a[2] += fs * fs;
    a[3] += S[0];
    a[4] += S[1];
    a[5] += fcm;
    a[6] += fcm * fcm;
    a[7] += S[2];
    a[8] += S[3];
    a[9] += c2;
    a[10] += c2 * c2;
    a[11] += S[4];
    a[12] += S[5];
    a[13] += S[6];
}

void launch_corr_sample(const DevState &d, const long long *X, const CorrDev &c, const CorrPairs &p, cudaStream_t st)
{
    if (p.n <= 0) return;
    corr_chunk_kernel<<<dim3(c.n_chunks, p.n), 256, 0, st>>>(d, X, c, p);
    corr_finish_kernel<<<p.n * d.n_rep, 128, 0, st>>>(d, c, p);
}

// S(q) of one (replica, wavevector) per block: the sums of cos and sin of
// q . x over the replica's atoms (x = q_fixed h, in [0, L)), each thread in
// ascending order, then a fixed tree; out = (C^2 + S^2) / N (Eq. sq with the
// i = j terms included).
__global__ void __launch_bounds__(256) sq_kernel(DevState d, const long long *X, const double *qv, int n_q,
                                                 double *out)
{
    const int r = blockIdx.y, k = blockIdx.x;
    const RepInfo ri = d.rep[r];
    const double qx = qv[3 * k], qy = qv[3 * k + 1], qz = qv[3 * k + 2];
    double c = 0.0, sn = 0.0;
    for (int i = threadIdx.x; i < ri.n_sites; i += 256) {
        const long long *x = X + 3 * (size_t)(ri.site_off + i);
        const double ph = qx * ((double)(uint32_t)x[0] * ri.h) + qy * ((double)(uint32_t)x[1] * ri.h) +
                          qz * ((double)(uint32_t)x[2] * ri.h);
        double sv, cv;
        sincos(ph, &sv, &cv);
        c = __dadd_rn(c, cv);
        sn = __dadd_rn(sn, sv);
    }
    __shared__ double rc[256], rs[256];
    rc[threadIdx.x] = c;
    rs[threadIdx.x] = sn;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            rc[threadIdx.x] = __dadd_rn(rc[threadIdx.x], rc[threadIdx.x + w]);
            rs[threadIdx.x] = __dadd_rn(rs[threadIdx.x], rs[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)r * n_q + k] = (rc[0] * rc[0] + rs[0] * rs[0]) / (double)ri.n_sites;
}

void launch_sq(const DevState &d, const long long *X, const double *qv, int n_q, double *out, cudaStream_t st)
{
    sq_kernel<<<dim3(n_q, d.n_rep), 256, 0, st>>>(d, X, qv, n_q, out);
}

// Pair-distance histogram of one replica (Eq. gr): every pair once, by the
// ring order: thread i takes the pairs (i, i + k mod N) for k = 1 .. (N-1)/2,
// and for even N the pair (i, i + N/2) when i < N/2.  Bin = floor(r / dr)
// with r from the FP64 minimum-image distance (each operation rounded once,
// in a fixed order), counted when below n_bins.
__global__ void __launch_bounds__(128) pair_hist_kernel(DevState d, const long long *X, double dr, int n_bins,
                                                        unsigned long long *counts)
{
    extern __shared__ unsigned int hist[];
    const int r = blockIdx.y;
    const RepInfo ri = d.rep[r];
    const int N = ri.n_sites;
    for (int b = threadIdx.x; b < n_bins; b += 128) hist[b] = 0;
    __syncthreads();
    const int i = blockIdx.x * 128 + threadIdx.x;
    if (blockIdx.x * 128 < N) {
        const double rmax = dr * (double)n_bins;
        const double guard2 = rmax * rmax * (1.0 + 1e-12);
        const int half = (N - 1) / 2;
        const bool extra = (N % 2 == 0) && i < N / 2;
        if (i < N) {
            const long long *xi = X + 3 * (size_t)(ri.site_off + i);
            const uint32_t ax = (uint32_t)xi[0], ay = (uint32_t)xi[1], az = (uint32_t)xi[2];
            for (int k = 1; k <= half + (extra ? 1 : 0); ++k) {
                int j = i + k;
                if (j >= N) j -= N;
                const long long *xj = X + 3 * (size_t)(ri.site_off + j);
                const double r2 = r2_fixed64((int)((uint32_t)xj[0] - ax), (int)((uint32_t)xj[1] - ay),
                                             (int)((uint32_t)xj[2] - az), ri.h);
                if (!(r2 < guard2)) continue;
                const int bin = (int)floor(__ddiv_rn(__dsqrt_rn(r2), dr));
                if (bin < n_bins) atomicAdd(&hist[bin], 1u);
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < n_bins; b += 128)
        if (hist[b]) atomicAdd(counts + (size_t)r * n_bins + b, (unsigned long long)hist[b]);
}

void launch_pair_hist(const DevState &d, const long long *X, int max_sites, double dr, int n_bins,
                      unsigned long long *counts, cudaStream_t st)
{
    pair_hist_kernel<<<dim3((max_sites + 127) / 128, d.n_rep), 128, sizeof(unsigned int) * n_bins, st>>>(
        d, X, dr, n_bins, counts);
}

void launch_gather(const DevState &d, int buf, long long *X, int *types, cudaStream_t st)
{
    gather_kernel<<<(d.n_sites + 255) / 256, 256, 0, st>>>(d, buf, X, types);
}

void launch_set_t0(const DevState &d, const long long *X, const int *types, const ObsState &o, cudaStream_t st)
{
    const int nm = d.n_sites / 3;
    set_t0_kernel<<<(nm + 127) / 128, 128, 0, st>>>(d, X, types, o);
}

void launch_observables(const DevState &d, const long long *X, const ObsState &o, const double *qa, int nqa,
                        const double *qc, int nqc, double *fs_site, double *fscm_mol, double *c2_mol, double *out,
                        cudaStream_t st)
{
    const int nm = d.n_sites / 3;
    observables_kernel<<<(nm + 127) / 128, 128, 0, st>>>(d, X, o, qa, nqa, qc, nqc, fs_site, fscm_mol, c2_mol);
    replica_sum_kernel<<<d.n_rep, 256, 0, st>>>(d, fs_site, 0, 1.0, out, 3, 0);
    replica_sum_kernel<<<d.n_rep, 256, 0, st>>>(d, fscm_mol, 1, 1.0, out, 3, 1);
    replica_sum_kernel<<<d.n_rep, 256, 0, st>>>(d, c2_mol, 1, 1.0, out, 3, 2);
}

}  // namespace flipmc
