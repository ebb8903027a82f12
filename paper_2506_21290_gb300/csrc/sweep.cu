// Checkerboard Metropolis sweep (arXiv 2506.21290 Sec. II.B on a cell grid).
//
// One warp owns one active cell of the current colour.  It stages the atoms of
// the cell and of its neighbour cells (27, or the 8 distinct cells when n_c = 2)
// in shared memory, draws the random numbers of all its attempts up front
// (Philox is counter-based: the draws do not depend on the state), then runs
// the cell's n attempts in order.  Every attempt spreads its candidate atoms
// over the 32 lanes, reduces Delta E with shuffles, decides, and commits in
// shared memory; the cell is written back to global memory at the end.
//
// Precision modes:
//   FP64: every Delta E is the FP64 ordered sum (moved atom ascending, then
//         partner index ascending) of the nonzero pair terms, evaluated with
//         unfused round-to-nearest operations; this reproduces the reference
//         FP64 chain exactly.
//   FP32: pair terms in FP32 from cell-local coordinates; the Metropolis
//         comparison against the FP64 threshold -T ln u is retaken in the FP64
//         ordered sum whenever |dE32 - thr| <= gap * (sum of term magnitudes),
//         or when a bond comes near its FENE divergence.
#include <algorithm>
#include <cstdio>

#include "cell_list.h"
#include "flipmc_device.cuh"

namespace flipmc {

constexpr int TERM_CAP = 192;       // nonzero FP64 terms of one move
constexpr unsigned FULL = 0xffffffffu;

struct PosF {
    float x, y, z;
};

// per-warp shared-memory scratch
struct Scratch {
    int4 *rec;              // [cap] staged records
    float4 *pos;            // [cap] cell-local FP32 positions (FP32 mode)
    unsigned long long *key; // [TERM_CAP]
    double *val;            // [TERM_CAP]
    double *sorted;         // [TERM_CAP]
    uint32_t *rnd;          // [32 * 8]
    double *thr;            // [32]
    int *cstart;            // [32]
    int *coff;              // [32]
    int *misc;              // [8]
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t scratch_bytes(int cap)
{
    return align16(sizeof(int4) * cap) + align16(sizeof(float4) * cap) +
           align16(sizeof(unsigned long long) * TERM_CAP) + 2 * align16(sizeof(double) * TERM_CAP) +
           align16(sizeof(uint32_t) * 256) + align16(sizeof(double) * 32) + 3 * align16(sizeof(int) * 32);
}

__device__ inline Scratch carve(unsigned char *base, int cap)
{
    Scratch s;
    size_t o = 0;
    s.rec = (int4 *)(base + o);
    o += align16(sizeof(int4) * cap);
    s.pos = (float4 *)(base + o);
    o += align16(sizeof(float4) * cap);
    s.key = (unsigned long long *)(base + o);
    o += align16(sizeof(unsigned long long) * TERM_CAP);
    s.val = (double *)(base + o);
    o += align16(sizeof(double) * TERM_CAP);
    s.sorted = (double *)(base + o);
    o += align16(sizeof(double) * TERM_CAP);
    s.rnd = (uint32_t *)(base + o);
    o += align16(sizeof(uint32_t) * 256);
    s.thr = (double *)(base + o);
    o += align16(sizeof(double) * 32);
    s.cstart = (int *)(base + o);
    o += align16(sizeof(int) * 32);
    s.coff = (int *)(base + o);
    o += align16(sizeof(int) * 32);
    s.misc = (int *)(base + o);
    return s;
}

// A proposed move, as the FP64 ordered sum needs it.
struct Move {
    int n;                 // atoms written (1..3), site indices ascending
    int site[3];
    int mol;
    uint32_t qo[3][3];     // old positions
    uint32_t qn[3][3];     // new positions
    int to[3], tn[3];      // old / new types
    bool moves_pos;
    bool intra;            // rotation: intramolecular pairs change too
};

__device__ __forceinline__ float r2_loc(const float4 &p, const PosF &s)
{
    const float dx = p.x - s.x, dy = p.y - s.y, dz = p.z - s.z;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

__device__ __forceinline__ float r2_int32f(uint32_t ax, uint32_t ay, uint32_t az, const uint32_t *b, float hf)
{
    const float dx = (float)(int)(ax - b[0]) * hf;
    const float dy = (float)(int)(ay - b[1]) * hf;
    const float dz = (float)(int)(az - b[2]) * hf;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// FP64 ordered Delta E of a move (all lanes return the same value).
// Returns MC_ST_EVALUATED or MC_ST_BOND_BREAK.
// ---------------------------------------------------------------------------
__device__ int dE64_ordered(const Move &mv, const Scratch &ws, int K, const ModelDev &md, double h, float hf,
                            float pre_r2, int lane, int *err, double &dE)
{
    if (lane == 0) ws.misc[0] = 0;
    __syncwarp();
    int brk = 0;
    for (int c = lane; c < K; c += 32) {
        const int4 r = ws.rec[c];
        const int sj = rec_site(r.w);
        bool in_set = false;
        for (int k = 0; k < mv.n; ++k) in_set |= (sj == mv.site[k]);
        if (in_set) continue;
        const bool bonded = rec_mol(r.w) == mv.mol;
        const int tj = rec_type(r.w);
        for (int k = 0; k < mv.n; ++k) {
            const int dxo = (int)((uint32_t)r.x - mv.qo[k][0]);
            const int dyo = (int)((uint32_t)r.y - mv.qo[k][1]);
            const int dzo = (int)((uint32_t)r.z - mv.qo[k][2]);
            const int dxn = (int)((uint32_t)r.x - mv.qn[k][0]);
            const int dyn = (int)((uint32_t)r.y - mv.qn[k][1]);
            const int dzn = (int)((uint32_t)r.z - mv.qn[k][2]);
            if (!bonded) {
                // conservative FP32 screen: a pair beyond every cutoff adds exactly 0
                const float fxo = (float)dxo * hf, fyo = (float)dyo * hf, fzo = (float)dzo * hf;
                const float fxn = (float)dxn * hf, fyn = (float)dyn * hf, fzn = (float)dzn * hf;
                const float r2of = fxo * fxo + fyo * fyo + fzo * fzo;
                const float r2nf = fxn * fxn + fyn * fyn + fzn * fzn;
                if (r2of > pre_r2 && r2nf > pre_r2) continue;
            }
            const double r2o = r2_fixed64(dxo, dyo, dzo, h);
            const double r2n = mv.moves_pos ? r2_fixed64(dxn, dyn, dzn, h) : r2o;
            const int abo = 3 * mv.to[k] + tj, abn = 3 * mv.tn[k] + tj;
            if (bonded && !(r2n < md.R2[abn])) brk = 1;
            const double term = __dsub_rn(phi64(md, r2n, abn, bonded), phi64(md, r2o, abo, bonded));
            if (term != 0.0) {
                const int p = atomicAdd(ws.misc, 1);
                if (p < TERM_CAP) {
                    ws.key[p] = ((unsigned long long)k << 32) | (unsigned)sj;
                    ws.val[p] = term;
                }
            }
        }
    }
    if (mv.intra && lane == 0) {
        const int pk[3] = {0, 0, 1}, pl[3] = {1, 2, 2};
        for (int pr = 0; pr < 3; ++pr) {
            const int k = pk[pr], l = pl[pr];
            const int ab = 3 * mv.to[k] + mv.to[l];
            const double r2o = r2_fixed64((int)(mv.qo[l][0] - mv.qo[k][0]), (int)(mv.qo[l][1] - mv.qo[k][1]),
                                          (int)(mv.qo[l][2] - mv.qo[k][2]), h);
            const double r2n = r2_fixed64((int)(mv.qn[l][0] - mv.qn[k][0]), (int)(mv.qn[l][1] - mv.qn[k][1]),
                                          (int)(mv.qn[l][2] - mv.qn[k][2]), h);
            if (!(r2n < md.R2[ab])) brk = 1;
            const double term = __dsub_rn(phi64(md, r2n, ab, true), phi64(md, r2o, ab, true));
            if (term != 0.0) {
                const int p = atomicAdd(ws.misc, 1);
                if (p < TERM_CAP) {
                    ws.key[p] = (3ull << 32) | (unsigned)pr;
                    ws.val[p] = term;
                }
            }
        }
    }
    brk = __any_sync(FULL, brk);
    __syncwarp();
    const int nt = ws.misc[0];
    if (nt > TERM_CAP) {
        if (lane == 0) atomicOr(err, ERR_TERMS);
        dE = __longlong_as_double(0x7FF8000000000000ll);
        return MC_ST_EVALUATED;
    }
    for (int e = lane; e < nt; e += 32) {
        const unsigned long long key = ws.key[e];
        int rank = 0;
        for (int f = 0; f < nt; ++f) rank += ws.key[f] < key;
        ws.sorted[rank] = ws.val[e];
    }
    __syncwarp();
    double s = 0.0;
    if (lane == 0)
        for (int e = 0; e < nt; ++e) s = __dadd_rn(s, ws.sorted[e]);
    dE = __shfl_sync(FULL, s, 0);
    __syncwarp();
    return brk ? MC_ST_BOND_BREAK : MC_ST_EVALUATED;
}

// ---------------------------------------------------------------------------
// FP32 Delta E loops.  Return (dE, mag, guard) reduced over the warp.
// SMALL: n_c = 2, candidates are distinct atoms and distances come from the
// int32 differences; otherwise from the cell-local float coordinates.
// ---------------------------------------------------------------------------
struct Acc32 {
    float dE, mag;
    int guard;
};

template <bool SMALL>
__device__ Acc32 atom_dE32(const Scratch &ws, int K, const ModelDev &md, int wi, int ti, const PosF &so,
                           const PosF &sn, const uint32_t *qo, const uint32_t *qn, float hf, float rc2max, int lane)
{
    const int mol = rec_mol(wi);
    float dE = 0.f, mag = 0.f;
    int guard = 0;
    for (int c = lane; c < K; c += 32) {
        float r2o, r2n;
        int wj;
        if (SMALL) {
            const int4 r = ws.rec[c];
            wj = r.w;
            r2o = r2_int32f((uint32_t)r.x, (uint32_t)r.y, (uint32_t)r.z, qo, hf);
            r2n = r2_int32f((uint32_t)r.x, (uint32_t)r.y, (uint32_t)r.z, qn, hf);
        } else {
            const float4 p = ws.pos[c];
            wj = __float_as_int(p.w);
            r2o = r2_loc(p, so);
            r2n = r2_loc(p, sn);
        }
        const bool bonded = rec_mol(wj) == mol;
        if ((r2o < rc2max || r2n < rc2max || bonded) && wj != wi) {
            const int ab = 3 * ti + rec_type(wj);
            float uo = 0.f, mo = 0.f, un = 0.f, mn = 0.f;
            if (r2o < md.rc2f[ab]) wca32(md, r2o, ab, uo, mo);
            if (r2n < md.rc2f[ab]) wca32(md, r2n, ab, un, mn);
            if (bonded) {
                if (r2n * md.invR2f[ab] >= md.bond_guard_f || r2o * md.invR2f[ab] >= md.bond_guard_f) {
                    guard = 1;
                } else {
                    float fo, fmo, fn, fmn;
                    fene32(md, r2o, ab, fo, fmo);
                    fene32(md, r2n, ab, fn, fmn);
                    uo += fo;
                    un += fn;
                    mo += fmo;
                    mn += fmn;
                }
            }
            dE += un - uo;
            mag += mo + mn;
        }
    }
    Acc32 a;
    a.dE = warp_sum_f(dE);
    a.mag = warp_sum_f(mag);
    a.guard = __any_sync(FULL, guard);
    return a;
}

template <bool SMALL>
__device__ Acc32 flip_dE32(const Scratch &ws, int K, const ModelDev &md, int mol, int wp2, int wq2, int tp, int tq,
                           const PosF &sp, const PosF &sq, const uint32_t *qp, const uint32_t *qq, float hf,
                           float rc2max, int lane)
{
    float dE = 0.f, mag = 0.f;
    int guard = 0;
    for (int c = lane; c < K; c += 32) {
        float r2p, r2q;
        int wj;
        if (SMALL) {
            const int4 r = ws.rec[c];
            wj = r.w;
            r2p = r2_int32f((uint32_t)r.x, (uint32_t)r.y, (uint32_t)r.z, qp, hf);
            r2q = r2_int32f((uint32_t)r.x, (uint32_t)r.y, (uint32_t)r.z, qq, hf);
        } else {
            const float4 p = ws.pos[c];
            wj = __float_as_int(p.w);
            r2p = r2_loc(p, sp);
            r2q = r2_loc(p, sq);
        }
        const int w2 = (int)((uint32_t)wj >> 2);
        const bool bonded = rec_mol(wj) == mol;
        if ((r2p < rc2max || r2q < rc2max || bonded) && w2 != wp2 && w2 != wq2) {
            const int tj = rec_type(wj);
            // atom p: type tp -> tq; atom q: type tq -> tp
            const int ab_po = 3 * tp + tj, ab_pn = 3 * tq + tj;
            const int ab_qo = 3 * tq + tj, ab_qn = 3 * tp + tj;
            float uo = 0.f, mo = 0.f, un = 0.f, mn = 0.f, u, m;
            if (r2p < md.rc2f[ab_po]) { wca32(md, r2p, ab_po, u, m); uo += u; mo += m; }
            if (r2p < md.rc2f[ab_pn]) { wca32(md, r2p, ab_pn, u, m); un += u; mn += m; }
            if (r2q < md.rc2f[ab_qo]) { wca32(md, r2q, ab_qo, u, m); uo += u; mo += m; }
            if (r2q < md.rc2f[ab_qn]) { wca32(md, r2q, ab_qn, u, m); un += u; mn += m; }
            if (bonded) {
                const float g = md.bond_guard_f;
                if (r2p * md.invR2f[ab_po] >= g || r2p * md.invR2f[ab_pn] >= g || r2q * md.invR2f[ab_qo] >= g ||
                    r2q * md.invR2f[ab_qn] >= g) {
                    guard = 1;
                } else {
                    fene32(md, r2p, ab_po, u, m); uo += u; mo += m;
                    fene32(md, r2p, ab_pn, u, m); un += u; mn += m;
                    fene32(md, r2q, ab_qo, u, m); uo += u; mo += m;
                    fene32(md, r2q, ab_qn, u, m); un += u; mn += m;
                }
            }
            dE += un - uo;
            mag += mo + mn;
        }
    }
    Acc32 a;
    a.dE = warp_sum_f(dE);
    a.mag = warp_sum_f(mag);
    a.guard = __any_sync(FULL, guard);
    return a;
}

template <bool SMALL>
__device__ Acc32 mol_dE32(const Scratch &ws, int K, const ModelDev &md, int mol, const int *t3, const PosF *so,
                          const PosF *sn, const uint32_t (*qo)[3], const uint32_t (*qn)[3], float hf, float rc2max,
                          int lane)
{
    float dE = 0.f, mag = 0.f;
    for (int c = lane; c < K; c += 32) {
        float r2o[3], r2n[3];
        int wj;
        if (SMALL) {
            const int4 r = ws.rec[c];
            wj = r.w;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                r2o[k] = r2_int32f((uint32_t)r.x, (uint32_t)r.y, (uint32_t)r.z, qo[k], hf);
                r2n[k] = r2_int32f((uint32_t)r.x, (uint32_t)r.y, (uint32_t)r.z, qn[k], hf);
            }
        } else {
            const float4 p = ws.pos[c];
            wj = __float_as_int(p.w);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                r2o[k] = r2_loc(p, so[k]);
                r2n[k] = r2_loc(p, sn[k]);
            }
        }
        if (rec_mol(wj) == mol) continue;
        bool near = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) near |= (r2o[k] < rc2max) | (r2n[k] < rc2max);
        if (!near) continue;
        const int tj = rec_type(wj);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int ab = 3 * t3[k] + tj;
            float u, m;
            if (r2o[k] < md.rc2f[ab]) { wca32(md, r2o[k], ab, u, m); dE -= u; mag += m; }
            if (r2n[k] < md.rc2f[ab]) { wca32(md, r2n[k], ab, u, m); dE += u; mag += m; }
        }
    }
    Acc32 a;
    a.dE = warp_sum_f(dE);
    a.mag = warp_sum_f(mag);
    a.guard = 0;
    return a;
}

// Rotation proposal about the centroid (FP64, unfused, the reference order).
__device__ void rotate_molecule(const uint32_t (*q)[3], uint32_t (*qn)[3], const uint32_t *w3, double rot_a, double h,
                                double inv_h)
{
    double rel[3][3], cen[3];
    for (int k = 0; k < 3; ++k)
        for (int ax = 0; ax < 3; ++ax) rel[k][ax] = __dmul_rn((double)(int)(q[k][ax] - q[0][ax]), h);
    for (int ax = 0; ax < 3; ++ax) cen[ax] = __ddiv_rn(__dadd_rn(__dadd_rn(rel[0][ax], rel[1][ax]), rel[2][ax]), 3.0);
    const double vw = 1.0;
    double v[3];
    for (int k = 0; k < 3; ++k)
        v[k] = __dmul_rn(rot_a, __dsub_rn(__dmul_rn(__dadd_rn((double)w3[k], 0.5), 0x1p-31), 1.0));
    const double vx = v[0], vy = v[1], vz = v[2];
    const double ww = __dmul_rn(vw, vw), xx = __dmul_rn(vx, vx), yy = __dmul_rn(vy, vy), zz = __dmul_rn(vz, vz);
    const double xy = __dmul_rn(vx, vy), xz = __dmul_rn(vx, vz), yz = __dmul_rn(vy, vz);
    const double wx = __dmul_rn(vw, vx), wy = __dmul_rn(vw, vy), wz = __dmul_rn(vw, vz);
    const double n2 = __dadd_rn(__dadd_rn(__dadd_rn(ww, xx), yy), zz);
    double R[3][3];
    R[0][0] = __ddiv_rn(__dsub_rn(__dsub_rn(__dadd_rn(ww, xx), yy), zz), n2);
    R[0][1] = __ddiv_rn(__dmul_rn(2.0, __dsub_rn(xy, wz)), n2);
    R[0][2] = __ddiv_rn(__dmul_rn(2.0, __dadd_rn(xz, wy)), n2);
    R[1][0] = __ddiv_rn(__dmul_rn(2.0, __dadd_rn(xy, wz)), n2);
    R[1][1] = __ddiv_rn(__dsub_rn(__dadd_rn(__dsub_rn(ww, xx), yy), zz), n2);
    R[1][2] = __ddiv_rn(__dmul_rn(2.0, __dsub_rn(yz, wx)), n2);
    R[2][0] = __ddiv_rn(__dmul_rn(2.0, __dsub_rn(xz, wy)), n2);
    R[2][1] = __ddiv_rn(__dmul_rn(2.0, __dadd_rn(yz, wx)), n2);
    R[2][2] = __ddiv_rn(__dadd_rn(__dsub_rn(__dsub_rn(ww, xx), yy), zz), n2);
    for (int k = 0; k < 3; ++k) {
        double p[3];
        for (int ax = 0; ax < 3; ++ax) p[ax] = __dsub_rn(rel[k][ax], cen[ax]);
        for (int ax = 0; ax < 3; ++ax) {
            const double np = __dadd_rn(
                __dadd_rn(__dadd_rn(__dmul_rn(R[ax][0], p[0]), __dmul_rn(R[ax][1], p[1])), __dmul_rn(R[ax][2], p[2])),
                cen[ax]);
            const long long nq = (long long)floor(__dadd_rn(__dmul_rn(np, inv_h), 0.5));
            qn[k][ax] = q[0][ax] + (uint32_t)nq;
        }
    }
}

// ---------------------------------------------------------------------------
// The phase kernel
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(128) phase_kernel(DevState d, int buf, int colour, LogArgs lg)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ModelDev md;
    __shared__ MixDev mx;
    {
        const int *src = (const int *)d.model;
        int *dst = (int *)&md;
        for (int i = threadIdx.x; i < (int)(sizeof(ModelDev) / 4); i += blockDim.x) dst[i] = src[i];
        const int *src2 = (const int *)d.mix;
        int *dst2 = (int *)&mx;
        for (int i = threadIdx.x; i < (int)(sizeof(MixDev) / 4); i += blockDim.x) dst2[i] = src2[i];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int g = blockIdx.x * (blockDim.x >> 5) + wib;
    if (g >= d.n_act) return;
    const int cap = d.stencil_cap;
    const Scratch ws = carve(smem + (size_t)wib * scratch_bytes(cap), cap);

    // ---- which cell ----
    const int r = find_segment(d.act_off, d.n_rep, g);
    const RepInfo ri = d.rep[r];
    const RepParam dy = d.par[r];
    const RepCtr ct = d.ctr[r];
    const int nc = ri.nc, h2 = nc >> 1;
    const int a_loc = g - d.act_off[r];
    const int cx = 2 * (a_loc % h2) + (colour & 1);
    const int cy = 2 * ((a_loc / h2) % h2) + ((colour >> 1) & 1);
    const int cz = 2 * (a_loc / (h2 * h2)) + ((colour >> 2) & 1);
    const int cellL = (cz * nc + cy) * nc + cx;
    const int cellG = ri.cell_off + cellL;
    const bool small = nc == 2;
    const int ns = small ? 8 : 27;

    // ---- stage the neighbourhood: own cell first ----
    int cnt = 0, cst = 0;
    if (lane < ns) {
        int ox, oy, oz;
        if (small) {
            ox = lane & 1; oy = (lane >> 1) & 1; oz = lane >> 2;
        } else {
            const int k = (lane == 0) ? 13 : (lane <= 13 ? lane - 1 : lane);   // 13 = (0,0,0)
            ox = k % 3 - 1; oy = (k / 3) % 3 - 1; oz = k / 9 - 1;
        }
        const int nx = (cx + ox + nc) % nc, ny = (cy + oy + nc) % nc, nz = (cz + oz + nc) % nc;
        const int c = ri.cell_off + (nz * nc + ny) * nc + nx;
        cst = d.cell_start[c];
        cnt = d.cell_start[c + 1] - cst;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const int K = __shfl_sync(FULL, incl, 31);
    const int n = __shfl_sync(FULL, cnt, 0);
    const int own_start = __shfl_sync(FULL, cst, 0);
    if (K > cap) {
        if (lane == 0) {
            atomicOr(d.err, ERR_STENCIL);
            d.cell_dE[cellG] = 0.0;
        }
        return;
    }
    if (lane < ns) {
        ws.cstart[lane] = cst;
        ws.coff[lane] = incl - cnt;
    }
    if (lane == 0) ws.coff[ns] = K;
    __syncwarp();

    // cell-local frame for FP32 coordinates: the cell centre
    const uint32_t P[3] = {
        (uint32_t)(((uint64_t)(2 * cx + 1) << 32) / (uint64_t)(2 * nc)) - ct.shift[0],
        (uint32_t)(((uint64_t)(2 * cy + 1) << 32) / (uint64_t)(2 * nc)) - ct.shift[1],
        (uint32_t)(((uint64_t)(2 * cz + 1) << 32) / (uint64_t)(2 * nc)) - ct.shift[2]};
    const float hf = ri.hf;
    auto local = [&](uint32_t x, uint32_t y, uint32_t z) {
        PosF p;
        p.x = (float)(int)(x - P[0]) * hf;
        p.y = (float)(int)(y - P[1]) * hf;
        p.z = (float)(int)(z - P[2]) * hf;
        return p;
    };
    const int4 *src = d.rec[buf];
    for (int idx = lane; idx < K; idx += 32) {
        const int k = find_segment(ws.coff, ns, idx);
        const int4 rc = src[ws.cstart[k] + (idx - ws.coff[k])];
        ws.rec[idx] = rc;
        if (PREC == MC_PREC_FP32 && !small) {
            const PosF p = local((uint32_t)rc.x, (uint32_t)rc.y, (uint32_t)rc.z);
            ws.pos[idx] = make_float4(p.x, p.y, p.z, __int_as_float(rc.w));
        }
    }
    __syncwarp();

    float rc2max = 0.f;
    for (int k = 0; k < 9; ++k) rc2max = fmaxf(rc2max, md.rc2f[k]);
    const float pre_r2 = rc2max * 1.01f;
    const double T = dy.T;
    const double gap = (double)md.recheck_gap_f;

    unsigned att[4] = {0, 0, 0, 0}, acc[4] = {0, 0, 0, 0};
    unsigned rej_geom = 0, rej_bond = 0, rechecks = 0;
    unsigned long long pairs = 0;
    double dE_cell = 0.0;

    for (int a0 = 0; a0 < n; a0 += 32) {
        // random numbers and thresholds of attempts a0 .. a0+31
        {
            const int a = a0 + lane;
            if (a < n) {
                const U4 b0 = rng_block((uint32_t)(2 * a), (uint32_t)cellL, ct.sweep, dy.seed);
                const U4 b1 = rng_block((uint32_t)(2 * a + 1), (uint32_t)cellL, ct.sweep, dy.seed);
                uint32_t *w = ws.rnd + 8 * lane;
                w[0] = b0.x; w[1] = b0.y; w[2] = b0.z; w[3] = b0.w;
                w[4] = b1.x; w[5] = b1.y; w[6] = b1.z; w[7] = b1.w;
                const unsigned long long u52 = ((unsigned long long)b0.z << 20) | (unsigned long long)(b0.w >> 12);
                const double u = __dmul_rn((double)(2ull * u52 + 1ull), 0x1p-53);
                ws.thr[lane] = -__dmul_rn(T, ln_series(u));
            }
        }
        __syncwarp();
        const int a_end = min(n, a0 + 32);
        for (int a = a0; a < a_end; ++a) {
            const uint32_t *w = ws.rnd + 8 * (a - a0);
            const double thr = ws.thr[a - a0];
            const int k = (int)(((unsigned long long)w[0] * (unsigned long long)n) >> 32);
            const int4 ri_rec = ws.rec[k];
            const int wi = ri_rec.w;
            const int mol = rec_mol(wi);
            const int mvt = move_type(w[1], mx);
            int status = MC_ST_EVALUATED;
            double dE = 0.0, dE64 = __longlong_as_double(0x7FF8000000000000ll);
            float scale = 0.f;
            int flags = 0;
            Move mv;
            mv.mol = mol;
            mv.intra = false;
            int kslot[3] = {k, -1, -1};
            att[mvt] += 1;

            if (mvt == MC_MOVE_ATOM) {
                mv.n = 1;
                mv.site[0] = rec_site(wi);
                mv.qo[0][0] = (uint32_t)ri_rec.x; mv.qo[0][1] = (uint32_t)ri_rec.y; mv.qo[0][2] = (uint32_t)ri_rec.z;
                for (int ax = 0; ax < 3; ++ax) mv.qn[0][ax] = mv.qo[0][ax] + (uint32_t)uniform_disp(w[4 + ax], dy.D_atom);
                mv.to[0] = mv.tn[0] = rec_type(wi);
                mv.moves_pos = true;
                if (cell_local(mv.qn[0][0], mv.qn[0][1], mv.qn[0][2], ct.shift, nc) != cellL) status = MC_ST_LEFT_CELL;
            } else if (mvt == MC_MOVE_FLIP) {
                const int axis = (int)(((unsigned long long)w[7] * 3ull) >> 32);
                const int sp = axis == 0 ? 1 : 0, sq = axis == 2 ? 1 : 2;
                int kp = -1, kq = -1;
                for (int j = lane; j < n; j += 32) {
                    const int wj = ws.rec[j].w;
                    if (rec_mol(wj) == mol) {
                        if (rec_slot(wj) == sp) kp = j;
                        if (rec_slot(wj) == sq) kq = j;
                    }
                }
                kp = __reduce_max_sync(FULL, kp);
                kq = __reduce_max_sync(FULL, kq);
                if (kp < 0 || kq < 0) {
                    status = MC_ST_NOT_IN_CELL;
                } else {
                    kslot[0] = kp; kslot[1] = kq;
                    const int4 rp = ws.rec[kp], rq = ws.rec[kq];
                    mv.n = 2;
                    mv.site[0] = rec_site(rp.w); mv.site[1] = rec_site(rq.w);
                    mv.qo[0][0] = mv.qn[0][0] = (uint32_t)rp.x; mv.qo[0][1] = mv.qn[0][1] = (uint32_t)rp.y;
                    mv.qo[0][2] = mv.qn[0][2] = (uint32_t)rp.z;
                    mv.qo[1][0] = mv.qn[1][0] = (uint32_t)rq.x; mv.qo[1][1] = mv.qn[1][1] = (uint32_t)rq.y;
                    mv.qo[1][2] = mv.qn[1][2] = (uint32_t)rq.z;
                    mv.to[0] = rec_type(rp.w); mv.to[1] = rec_type(rq.w);
                    mv.tn[0] = mv.to[1]; mv.tn[1] = mv.to[0];
                    mv.moves_pos = false;
                }
            } else {
                int ks[3] = {-1, -1, -1};
                for (int j = lane; j < n; j += 32) {
                    const int wj = ws.rec[j].w;
                    if (rec_mol(wj) == mol) ks[rec_slot(wj)] = j;
                }
                for (int s = 0; s < 3; ++s) ks[s] = __reduce_max_sync(FULL, ks[s]);
                if (ks[0] < 0 || ks[1] < 0 || ks[2] < 0) {
                    status = MC_ST_NOT_IN_CELL;
                } else {
                    mv.n = 3;
                    mv.moves_pos = true;
                    for (int s = 0; s < 3; ++s) {
                        kslot[s] = ks[s];
                        const int4 rs = ws.rec[ks[s]];
                        mv.site[s] = rec_site(rs.w);
                        mv.qo[s][0] = (uint32_t)rs.x; mv.qo[s][1] = (uint32_t)rs.y; mv.qo[s][2] = (uint32_t)rs.z;
                        mv.to[s] = mv.tn[s] = rec_type(rs.w);
                    }
                    if (mvt == MC_MOVE_MOL_TRANS) {
                        int32_t dd[3];
                        for (int ax = 0; ax < 3; ++ax) dd[ax] = uniform_disp(w[4 + ax], dy.D_mol);
                        for (int s = 0; s < 3; ++s)
                            for (int ax = 0; ax < 3; ++ax) mv.qn[s][ax] = mv.qo[s][ax] + (uint32_t)dd[ax];
                    } else {
                        rotate_molecule(mv.qo, mv.qn, w + 4, mx.rot_a, ri.h, ri.inv_h);
                        mv.intra = true;
                    }
                    for (int s = 0; s < 3; ++s)
                        if (cell_local(mv.qn[s][0], mv.qn[s][1], mv.qn[s][2], ct.shift, nc) != cellL)
                            status = MC_ST_LEFT_CELL;
                }
            }

            bool accept = false;
            if (status == MC_ST_EVALUATED) {
                if (PREC == MC_PREC_FP64) {
                    status = dE64_ordered(mv, ws, K, md, ri.h, hf, pre_r2, lane, d.err, dE);
                    dE64 = dE;
                    accept = status == MC_ST_EVALUATED && dE <= thr;
                    pairs += (unsigned long long)(2 * mv.n) * (unsigned long long)K;
                } else {
                    Acc32 acc32;
                    if (mvt == MC_MOVE_ATOM) {
                        const PosF so = local(mv.qo[0][0], mv.qo[0][1], mv.qo[0][2]);
                        const PosF sn = local(mv.qn[0][0], mv.qn[0][1], mv.qn[0][2]);
                        acc32 = small ? atom_dE32<true>(ws, K, md, wi, mv.to[0], so, sn, mv.qo[0], mv.qn[0], hf, rc2max, lane)
                                      : atom_dE32<false>(ws, K, md, wi, mv.to[0], so, sn, mv.qo[0], mv.qn[0], hf, rc2max, lane);
                        pairs += 2ull * (unsigned long long)K;
                    } else if (mvt == MC_MOVE_FLIP) {
                        const PosF sp = local(mv.qo[0][0], mv.qo[0][1], mv.qo[0][2]);
                        const PosF sq = local(mv.qo[1][0], mv.qo[1][1], mv.qo[1][2]);
                        const int wp2 = (int)((uint32_t)ws.rec[kslot[0]].w >> 2);
                        const int wq2 = (int)((uint32_t)ws.rec[kslot[1]].w >> 2);
                        acc32 = small ? flip_dE32<true>(ws, K, md, mol, wp2, wq2, mv.to[0], mv.to[1], sp, sq, mv.qo[0], mv.qo[1], hf, rc2max, lane)
                                      : flip_dE32<false>(ws, K, md, mol, wp2, wq2, mv.to[0], mv.to[1], sp, sq, mv.qo[0], mv.qo[1], hf, rc2max, lane);
                        pairs += 2ull * (unsigned long long)K;
                    } else {
                        PosF so[3], sn[3];
                        for (int s = 0; s < 3; ++s) {
                            so[s] = local(mv.qo[s][0], mv.qo[s][1], mv.qo[s][2]);
                            sn[s] = local(mv.qn[s][0], mv.qn[s][1], mv.qn[s][2]);
                        }
                        acc32 = small ? mol_dE32<true>(ws, K, md, mol, mv.to, so, sn, mv.qo, mv.qn, hf, rc2max, lane)
                                      : mol_dE32<false>(ws, K, md, mol, mv.to, so, sn, mv.qo, mv.qn, hf, rc2max, lane);
                        pairs += 6ull * (unsigned long long)K;
                        if (mv.intra) {
                            // intramolecular bonds change under rotation: add them (uniform on all lanes)
                            const int pk[3] = {0, 0, 1}, pl[3] = {1, 2, 2};
                            for (int pr = 0; pr < 3; ++pr) {
                                const int kk = pk[pr], ll = pl[pr];
                                const int ab = 3 * mv.to[kk] + mv.to[ll];
                                const float r2o = r2_int32f(mv.qo[ll][0], mv.qo[ll][1], mv.qo[ll][2], mv.qo[kk], hf);
                                const float r2n = r2_int32f(mv.qn[ll][0], mv.qn[ll][1], mv.qn[ll][2], mv.qn[kk], hf);
                                if (r2n * md.invR2f[ab] >= md.bond_guard_f || r2o * md.invR2f[ab] >= md.bond_guard_f) {
                                    acc32.guard = 1;
                                    continue;
                                }
                                float u, m;
                                if (r2o < md.rc2f[ab]) { wca32(md, r2o, ab, u, m); acc32.dE -= u; acc32.mag += m; }
                                if (r2n < md.rc2f[ab]) { wca32(md, r2n, ab, u, m); acc32.dE += u; acc32.mag += m; }
                                fene32(md, r2o, ab, u, m); acc32.dE -= u; acc32.mag += m;
                                fene32(md, r2n, ab, u, m); acc32.dE += u; acc32.mag += m;
                            }
                        }
                    }
                    dE = (double)acc32.dE;
                    scale = acc32.mag;
                    const double diff = fabs(dE - thr);
                    if (acc32.guard || !(diff > gap * (double)acc32.mag)) {
                        flags = 1;
                        rechecks += 1;
                        status = dE64_ordered(mv, ws, K, md, ri.h, hf, pre_r2, lane, d.err, dE64);
                        accept = status == MC_ST_EVALUATED && dE64 <= thr;
                    } else {
                        accept = dE <= thr;
                    }
                }
            }

            if (status == MC_ST_LEFT_CELL || status == MC_ST_NOT_IN_CELL) rej_geom += 1;
            if (status == MC_ST_BOND_BREAK) rej_bond += 1;
            if (accept) {
                acc[mvt] += 1;
                const double used = (PREC == MC_PREC_FP64 || flags) ? dE64 : dE;
                dE_cell = __dadd_rn(dE_cell, used);
                if (lane == 0) {
                    if (mvt == MC_MOVE_FLIP) {
                        int4 rp = ws.rec[kslot[0]], rq = ws.rec[kslot[1]];
                        rp.w = (rp.w & ~3) | mv.tn[0];
                        rq.w = (rq.w & ~3) | mv.tn[1];
                        ws.rec[kslot[0]] = rp;
                        ws.rec[kslot[1]] = rq;
                        if (PREC == MC_PREC_FP32 && !small) {
                            ws.pos[kslot[0]].w = __int_as_float(rp.w);
                            ws.pos[kslot[1]].w = __int_as_float(rq.w);
                        }
                    } else {
                        for (int s = 0; s < mv.n; ++s) {
                            int4 rs = ws.rec[kslot[s]];
                            rs.x = (int)mv.qn[s][0]; rs.y = (int)mv.qn[s][1]; rs.z = (int)mv.qn[s][2];
                            ws.rec[kslot[s]] = rs;
                            if (PREC == MC_PREC_FP32 && !small) {
                                const PosF p = local(mv.qn[s][0], mv.qn[s][1], mv.qn[s][2]);
                                ws.pos[kslot[s]] = make_float4(p.x, p.y, p.z, __int_as_float(rs.w));
                            }
                        }
                    }
                }
            }
            if (lg.base != nullptr && lane == 0) {
                const uint64_t sl = ct.sweep - lg.sweep0;
                mc_log_entry *e = lg.base + (size_t)ri.site_off * (size_t)lg.n_sweeps + (size_t)sl * (size_t)ri.n_sites +
                                  (size_t)(own_start - ri.site_off) + (size_t)a;
                e->site = rec_site(wi);
                e->move = (int16_t)mvt;
                e->flags = (int16_t)flags;
                e->status = status;
                e->accepted = accept ? 1 : 0;
                e->dE = status == MC_ST_EVALUATED ? dE : __longlong_as_double(0x7FF8000000000000ll);
                e->dE64 = dE64;
                e->scale = (double)scale;
            }
            __syncwarp();
        }
    }

    // ---- write back the cell; count periodic images crossed ----
    int4 *dst = d.rec[buf] + own_start;
    for (int k = lane; k < n; k += 32) {
        const int4 nw = ws.rec[k];
        const int4 od = dst[k];
        const int site = ri.site_off + rec_site(nw.w);
        const uint32_t o3[3] = {(uint32_t)od.x, (uint32_t)od.y, (uint32_t)od.z};
        const uint32_t n3[3] = {(uint32_t)nw.x, (uint32_t)nw.y, (uint32_t)nw.z};
        for (int ax = 0; ax < 3; ++ax) {
            const long long moved = (long long)o3[ax] + (long long)(int)(n3[ax] - o3[ax]);
            if (moved < 0) d.img[3 * site + ax] -= 1;
            else if (moved >= 4294967296ll) d.img[3 * site + ax] += 1;
        }
        dst[k] = nw;
    }
    if (lane == 0) {
        d.cell_dE[cellG] = dE_cell;
        unsigned long long *st = d.stats + (size_t)r * STAT_N;
        for (int m = 0; m < 4; ++m) {
            if (att[m]) atomicAdd(st + STAT_ATT + m, (unsigned long long)att[m]);
            if (acc[m]) atomicAdd(st + STAT_ACC + m, (unsigned long long)acc[m]);
        }
        if (rej_geom) atomicAdd(st + STAT_REJ_GEOM, (unsigned long long)rej_geom);
        if (rej_bond) atomicAdd(st + STAT_REJ_BOND, (unsigned long long)rej_bond);
        if (pairs) atomicAdd(st + STAT_PAIRS, pairs);
        if (rechecks) atomicAdd(st + STAT_RECHECK, (unsigned long long)rechecks);
    }
}

// Per replica: add the sweep's accepted Delta E (cells in a fixed reduction
// order, so the result is reproducible), count the sweep, advance the counter.
__global__ void __launch_bounds__(256) finalize_kernel(DevState d)
{
    const int r = blockIdx.x;
    const RepInfo ri = d.rep[r];
    const int ncell = ri.nc * ri.nc * ri.nc;
    double s = 0.0;
    for (int c = threadIdx.x; c < ncell; c += 256) s = __dadd_rn(s, d.cell_dE[ri.cell_off + c]);
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        d.e_run[r] = __dadd_rn(d.e_run[r], red[0]);
        d.stats[(size_t)r * STAT_N + STAT_SWEEPS] += 1;
        d.ctr[r].sweep += 1;
    }
}

size_t phase_smem_bytes(int stencil_cap, int warps_per_block)
{
    return scratch_bytes(stencil_cap) * (size_t)warps_per_block;
}

int phase_set_smem_limit(int stencil_cap, int warps_per_block)
{
    // the attribute is per kernel, shared by all handles: keep the largest request
    static int granted = 0;
    const int bytes = std::max(granted, (int)phase_smem_bytes(stencil_cap, warps_per_block));
    granted = bytes;
    cudaError_t e1 = cudaFuncSetAttribute(phase_kernel<MC_PREC_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaError_t e2 = cudaFuncSetAttribute(phase_kernel<MC_PREC_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return (e1 == cudaSuccess && e2 == cudaSuccess) ? 0 : -1;
}

void launch_colour_phases(const DevState &d, int buf, int warps_per_block, const LogArgs &lg, cudaStream_t st)
{
    const int blocks = (d.n_act + warps_per_block - 1) / warps_per_block;
    const size_t sm = phase_smem_bytes(d.stencil_cap, warps_per_block);
    for (int colour = 0; colour < 8; ++colour) {
        if (d.precision == MC_PREC_FP64)
            phase_kernel<MC_PREC_FP64><<<blocks, 32 * warps_per_block, sm, st>>>(d, buf, colour, lg);
        else
            phase_kernel<MC_PREC_FP32><<<blocks, 32 * warps_per_block, sm, st>>>(d, buf, colour, lg);
    }
}

void launch_finalize(const DevState &d, cudaStream_t st)
{
    finalize_kernel<<<d.n_rep, 256, 0, st>>>(d);
}

void launch_phases(const DevState &d, int buf, int warps_per_block, const LogArgs &lg, cudaStream_t st)
{
    launch_colour_phases(d, buf, warps_per_block, lg, st);
    launch_finalize(d, st);
}

}  // namespace flipmc
