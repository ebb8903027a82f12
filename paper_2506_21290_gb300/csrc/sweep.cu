// Checkerboard Metropolis sweep (arXiv 2506.21290 Sec. II.B on a cell grid).
//
// A group of W warps (W = 1, 2, 4 or 8) owns one active cell of the current
// colour.  It stages the raw records of the cell and of its neighbour cells
// (27, or the 8 distinct cells when n_c = 2) in shared memory, loaded from L2
// by all its lanes at once, and loads the draws of its attempts, which the
// cell-list build decoded beforehand (Philox is counter-based: the draws do
// not depend on the state).  The cell's n attempts then run in rounds: in a round the W warps
// evaluate W consecutive attempts against the same state, one attempt per
// warp.  The attempts commit in order up to the first one that an earlier
// accepted attempt of the round could have influenced: same molecule, or an
// atom of the earlier move (old or new position) within 1.01 times the largest
// WCA cutoff of an atom of the later one.  Interactions between different
// molecules are WCA only, so an attempt that passes this test has exactly the
// Delta E, decision and log entry it would have had after the earlier commit;
// the uncommitted attempts are evaluated again in the next round.  The chain is
// therefore the sequential one, for every W.
//
// One attempt, one warp (FP32 mode):
//   1. screen: each lane takes one candidate per 32-candidate step; the exact
//      int32 minimum-image differences to the moved atom's old position,
//      converted to FP32, give r^2, and the new one follows as
//      r'^2 = r^2 - 2 d.e + |e|^2; candidates inside the screening radius
//      (r^2 < 1.01 x the largest WCA cutoff squared), or in the same molecule,
//      are queued in ballot order.  Both modes run this pass.
//   2. interaction pass over the queue: WCA (Eq. 1) and FENE (Eq. 2), old and
//      new, in FP32 from the exact int32 differences (one rounding per axis),
//      each term with a magnitude m that bounds its rounding error.
//   3. decision: |dE32 - thr32| against gap * sum(m) (gap = 1e-5 by default)
//      plus the error bound of the FP32 threshold -T ln u.  The FP32 Delta E is
//      within 6.3e-6 sum(m) of the exact one (distances within ~9 units of
//      2^-24, each term's sensitivity to them at most 6 m, its own evaluation
//      ~31 units, the sums ~21 units), so outside that band the FP32
//      comparison agrees with the FP64 one; inside it (or near a FENE
//      divergence, or when the queue overflowed) the warp recomputes Delta E
//      and the threshold in FP64, in the reference order, and decides on them.
// No step of the hot path branches per lane: lanes past the staged atoms read
// a padding record, discarded queue writes go to a spare slot, and terms are
// masked instead of skipped.
//
// FP64 mode: every Delta E is the FP64 ordered sum (moved atom ascending, then
// partner index ascending) of the nonzero pair terms, each operation unfused
// and rounded to nearest, and the threshold is the FP64 series logarithm; this
// reproduces the reference FP64 chain exactly.  The terms are taken over the
// queued partners only: the screening radius exceeds every cutoff by far more
// than the FP32 distance error, so every partner with a nonzero term is queued.
#include <algorithm>
#include <cstdio>

#include "cell_list.h"
#include "cell_list_dev.cuh"
#include "flipmc_device.cuh"

namespace flipmc {

constexpr int TERM_CAP = 128;       // nonzero FP64 terms of one move
constexpr int QW = 64;              // interaction queue entries per warp
constexpr int BLOCK = 128;          // threads per block for W = 2, 4 and the persistent W = 1 kernel (and the per-replica sums)

// threads per block of the sweep kernels: BLOCK, or one group of W warps when W > 4
template <int W>
__host__ __device__ constexpr int block_threads() { return W > 4 ? 32 * W : BLOCK; }
constexpr unsigned FULL = 0xffffffffu;
constexpr int PADS = kPadSlots;     // padding candidates staged after the K atoms
constexpr int PAD_W = kPadWord;     // their record word: type 0, a molecule no atom has
constexpr int SCREEN_U = 4;         // largest number of 64-candidate steps per screening block
constexpr int SU = 2;               // record loads in flight per lane while staging

// ---------------------------------------------------------------------------
// packed FP32 pairs (f32x2, sm_100 and later)
// ---------------------------------------------------------------------------
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t pk(float a, float b)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2_t v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b)
{
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t mul2(f2_t a, f2_t b)
{
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c)
{
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

struct Q3 {
    uint32_t x, y, z;
};

// ---------------------------------------------------------------------------
// Distances from the raw fixed-point records.  The int32 difference of two
// 32-bit fixed-point coordinates is their minimum-image difference in units of
// the quantum h = L / 2^32, exactly, for any n_c.  Converting it to FP32 rounds
// once (relative 2^-24), so a squared distance carries only that rounding and
// the rounding of its squares and sums; no absolute error grows with the
// distance from any origin.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dq(uint32_t a, uint32_t b) { return (float)(int)(a - b); }

// squared distance of record r to position b, fixed-point units squared
__device__ __forceinline__ float r2_q(const int4 &r, const Q3 &b)
{
    const float x = dq((uint32_t)r.x, b.x), y = dq((uint32_t)r.y, b.y), z = dq((uint32_t)r.z, b.z);
    return fmaf(x, x, fmaf(y, y, z * z));
}

// squared distance in sigma units from raw fixed-point positions (one lane,
// intramolecular pairs of a rotation)
__device__ __forceinline__ float r2_int32f(const int4 &r, const Q3 b, float hf)
{
    const float dx = (float)(int)((uint32_t)r.x - b.x) * hf;
    const float dy = (float)(int)((uint32_t)r.y - b.y) * hf;
    const float dz = (float)(int)((uint32_t)r.z - b.z) * hf;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// a moved atom's position relative to the cell centre P, for the conflict test
struct PosH {
    float x, y, z;
};

// ---------------------------------------------------------------------------
// shared memory
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// Bulk copies global -> shared (cp.async.bulk) completing on an mbarrier: the
// staging of one-warp groups (W = 1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *mb)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n\tfence.proxy.async.shared::cta;" ::"r"(smem_u32(mb))
                 : "memory");
}

// the one arrival of a phase, announcing the bytes its copies will deliver
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *mb, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_done(uint64_t *mb, unsigned parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(mb)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from global to
// shared.  The proxy fence orders this group's earlier generic accesses to the
// destination before the copy's writes; the source was written before the
// last grid-wide barrier (or kernel boundary), or by a neighbour cell whose
// release the group acquired, and the copy reads it in L2.
__device__ __forceinline__ void bulk_to_smem(void *dst, const void *src, unsigned bytes, uint64_t *mb)
{
    asm volatile("fence.proxy.async.shared::cta;\n\t"
                 "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mb))
                 : "memory");
}

// per warp: interaction queue, and (aliased, used after it) the FP64 term buffers
struct WarpScr {
    int *qc;                    // [QW + 1] queued candidate indices, then a slot that takes discarded writes
    unsigned long long *key;    // [TERM_CAP] term keys; after ranking, the values in key order (as doubles)
    double *val;                // [TERM_CAP]
    int *cnt;                   // [4]
};

// the outcome of one evaluated attempt (registers of the evaluating warp,
// which also commits it)
struct Res {
    int status, accept, flags, mvt, nmv, site, mol;
    int ks[3], t3n[3];
    uint32_t qn[3][3];
    float dE32;                 // FP32 mode: the FP32 Delta E
    float scale;                // FP32 mode: sum of the term magnitudes
    double dE64;                // the FP64 Delta E (FP64 mode, or an FP32-mode recheck), else NaN
    int pairs;                  // site-pair evaluations per candidate (2 or 6)
    int inter;                  // this lane's pair-potential evaluations inside their range
};

// what the conflict test of the later attempts of a round reads (W > 1)
struct Near {
    int accept, mol, nat, pad;
    float px[6], py[6], pz[6];  // the move's atoms (old and new) relative to the cell centre, fixed-point units
};

// Attempt counts of one warp over one cell, one counter per lane: lane l
// counts stats slot l (l < TALLY_N: attempts and acceptances per move type,
// geometric and bond rejections, pair evaluations, rechecks).  Every lane
// holds the outcome of the attempt, so each adds to its own counter and a
// commit touches no memory for its counts.  Pair evaluations are counted per
// candidate (2 or 6) and scaled by the neighbourhood size K at the end.
constexpr int TALLY_N = 12;
static_assert(STAT_ATT == 0 && STAT_ACC == 4 && STAT_REJ_GEOM == 8 && STAT_REJ_BOND == 9 && STAT_PAIRS == 10 &&
                  STAT_RECHECK == 11,
              "lane l of a tally counts stats slot l");

// a warp's counts as the group combines them (W > 1)
struct Tally {
    unsigned cnt[TALLY_N];
    unsigned inter;             // pair-potential evaluations inside their range (summed over the warp's lanes)
    float dEf;                  // FP32 mode: accepted Delta E, in commit order
    double dE;                  // FP64 mode: accepted Delta E, in commit order
};

struct Group {
    int4 *rec;                  // [cap] raw records {qx, qy, qz, w} of the neighbourhood, own cell first,
                                //       then kPadSlots padding records
    uint64_t *mbar;             // completion barrier of the bulk copies that stage rec (W = 1)
    uint32_t *rnd;              // [32 * 8] random words of a chunk of attempts
    double *thr64;              // [32]
    float *thr32;               // [32]
    int *cstart;                // [32]
    int *coff;                  // [32]
    int *misc;                  // [32]
    Near *near;                 // [W]
    Tally *tally;               // [W] each warp's counts over the cell, combined at its end (W > 1)
    unsigned char *warp_base;   // W per-warp scratch blocks
};

enum { MS_K = 0, MS_N = 1, MS_START = 2, MS_PHASE = 3, MS_CLASH = 4 /* [W <= 8] */, MS_FAIL = 16 };

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ constexpr size_t warp_scr_bytes()
{
    return (al16(sizeof(int) * (QW + 1)) > al16(sizeof(unsigned long long) * TERM_CAP)
                ? al16(sizeof(int) * (QW + 1))
                : al16(sizeof(unsigned long long) * TERM_CAP)) +
           al16(sizeof(double) * TERM_CAP) + al16(sizeof(int) * 4);
}

// Layout of a group's shared memory: the fixed-size parts first (at offsets
// known at compile time for each W), the neighbourhood records last.
__host__ __device__ constexpr size_t group_fixed_bytes(int W)
{
    return 16 + al16(sizeof(uint32_t) * 256) + al16(sizeof(double) * 32) + al16(sizeof(float) * 32) +
           3 * al16(sizeof(int) * 32) + al16(sizeof(Near) * W) + al16(sizeof(Tally) * W) +
           (size_t)W * warp_scr_bytes();
}

__host__ __device__ inline size_t group_bytes(int cap, int W)
{
    return group_fixed_bytes(W) + al16(sizeof(int4) * cap);
}

__device__ inline Group carve(unsigned char *base, int W)
{
    Group s;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + o;
        o += al16(bytes);
        return p;
    };
    s.mbar = (uint64_t *)take(16);
    s.rnd = (uint32_t *)take(sizeof(uint32_t) * 256);
    s.thr64 = (double *)take(sizeof(double) * 32);
    s.thr32 = (float *)take(sizeof(float) * 32);
    s.cstart = (int *)take(sizeof(int) * 32);
    s.coff = (int *)take(sizeof(int) * 32);
    s.misc = (int *)take(sizeof(int) * 32);
    s.near = (Near *)take(sizeof(Near) * W);
    s.tally = (Tally *)take(sizeof(Tally) * W);
    s.warp_base = take((size_t)W * warp_scr_bytes());
    s.rec = (int4 *)(base + o);
    return s;
}

__device__ inline WarpScr warp_scr(const Group &G, int wig)
{
    unsigned char *b = G.warp_base + (size_t)wig * warp_scr_bytes();
    WarpScr s;
    const size_t q = al16(sizeof(int) * (QW + 1));
    const size_t k = al16(sizeof(unsigned long long) * TERM_CAP);
    const size_t qk = q > k ? q : k;
    s.qc = (int *)b;
    s.key = (unsigned long long *)b;    // aliases the queue: used only after it
    s.val = (double *)(b + qk);
    s.cnt = (int *)(b + qk + al16(sizeof(double) * TERM_CAP));
    return s;
}

// barrier over the 32 W threads of one cell group
template <int W>
__device__ __forceinline__ void gsync(int gid)
{
    if constexpr (W == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(32 * W) : "memory");
    }
}

__device__ __forceinline__ float warp_sum_f(float v)
{
    // butterfly: every lane ends with the same bits (each step adds the same pair)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// The staged raw records of the neighbourhood (shared memory), as the FP64
// ordered sum reads them.
struct RecView {
    const int4 *smem;
    __device__ int4 at(int c) const { return smem[c]; }
};

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

// ---------------------------------------------------------------------------
// FP64 ordered Delta E of a move, one warp (all lanes return the same value).
// Returns MC_ST_EVALUATED or MC_ST_BOND_BREAK.
// ---------------------------------------------------------------------------
// The candidates are the nq queued ones of the FP32 candidate pass when
// nq >= 0 (the queue holds every partner within the screening radius and every
// atom of the molecule, so no nonzero term is missed), else all K staged atoms.
// Terms are keyed by (moved atom, partner site), so which lane computes a term
// does not change the sum.
__device__ __noinline__ int dE64_ordered(const Move &mv, const RecView rv, const WarpScr S, int K, int nq,
                                         const ModelDev &md, double h, float hf, float pre_r2, int lane, int *err,
                                         double &dE, int &inter)
{
    inter = 0;
    static_assert(QW <= 64, "a lane takes at most two queue entries");
    // the term buffers alias the queue: take the entries into registers first
    int qe0 = -1, qe1 = -1;
    if (nq >= 0) {
        if (lane < nq) qe0 = S.qc[lane];
        if (lane + 32 < nq) qe1 = S.qc[lane + 32];
    }
    __syncwarp();
    if (lane == 0) S.cnt[0] = 0;
    __syncwarp();
    int brk = 0;
    auto term_of = [&](int c) {
        const int4 r = rv.at(c);
        const int sj = rec_site(r.w);
        bool in_set = false;
        for (int k = 0; k < mv.n; ++k) in_set |= (sj == mv.site[k]);
        if (in_set) return;
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
            inter += (r2o < md.rc2[abo]) + (r2n < md.rc2[abn]) + (bonded ? 2 : 0);
            if (bonded && !(r2n < md.R2[abn])) brk = 1;
            const double term = __dsub_rn(phi64(md, r2n, abn, bonded), phi64(md, r2o, abo, bonded));
            if (term != 0.0) {
                const int p = atomicAdd(S.cnt, 1);
                if (p < TERM_CAP) {
                    S.key[p] = ((unsigned long long)k << 32) | (unsigned)sj;
                    S.val[p] = term;
                }
            }
        }
    };
    if (nq >= 0) {
        if (qe0 >= 0) term_of(qe0);
        if (qe1 >= 0) term_of(qe1);
    } else {
        for (int c = lane; c < K; c += 32) term_of(c);
    }
    if (mv.intra && lane == 0) {
        const int pk3[3] = {0, 0, 1}, pl3[3] = {1, 2, 2};
        for (int pr = 0; pr < 3; ++pr) {
            const int k = pk3[pr], l = pl3[pr];
            const int ab = 3 * mv.to[k] + mv.to[l];
            const double r2o = r2_fixed64((int)(mv.qo[l][0] - mv.qo[k][0]), (int)(mv.qo[l][1] - mv.qo[k][1]),
                                          (int)(mv.qo[l][2] - mv.qo[k][2]), h);
            const double r2n = r2_fixed64((int)(mv.qn[l][0] - mv.qn[k][0]), (int)(mv.qn[l][1] - mv.qn[k][1]),
                                          (int)(mv.qn[l][2] - mv.qn[k][2]), h);
            inter += (r2o < md.rc2[ab]) + (r2n < md.rc2[ab]) + 2;
            if (!(r2n < md.R2[ab])) brk = 1;
            const double term = __dsub_rn(phi64(md, r2n, ab, true), phi64(md, r2o, ab, true));
            if (term != 0.0) {
                const int p = atomicAdd(S.cnt, 1);
                if (p < TERM_CAP) {
                    S.key[p] = (3ull << 32) | (unsigned)pr;
                    S.val[p] = term;
                }
            }
        }
    }
    brk = __any_sync(FULL, brk);
    __syncwarp();
    const int nt = S.cnt[0];
    if (nt > TERM_CAP) {
        if (lane == 0) atomicOr(err, ERR_TERMS);
        dE = __longlong_as_double(0x7FF8000000000000ll);
        return MC_ST_EVALUATED;
    }
    // rank every term by its key (keys are distinct), then put the values in
    // key order over the key array and sum them in that order
    static_assert(TERM_CAP <= 128, "a lane ranks at most four terms");
    unsigned long long kk[4];
    double vv[4];
    int rk[4] = {0, 0, 0, 0};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int e = lane + 32 * s;
        kk[s] = e < nt ? S.key[e] : ~0ull;
        vv[s] = e < nt ? S.val[e] : 0.0;
    }
    for (int f = 0; f < nt; ++f) {
        const unsigned long long kf = S.key[f];
#pragma unroll
        for (int s = 0; s < 4; ++s) rk[s] += kf < kk[s];
    }
    __syncwarp();
    double *sorted = (double *)S.key;
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (lane + 32 * s < nt) sorted[rk[s]] = vv[s];
    __syncwarp();
    double s = 0.0;
    if (lane == 0)
        for (int e = 0; e < nt; ++e) s = __dadd_rn(s, sorted[e]);
    dE = __shfl_sync(FULL, s, 0);
    __syncwarp();
    return brk ? MC_ST_BOND_BREAK : MC_ST_EVALUATED;
}

// Rotation proposal about the centroid (FP64, unfused, the reference order).
__device__ __noinline__ void rotate_molecule(const uint32_t (*q)[3], uint32_t (*qn)[3], const uint32_t *w3,
                                             double rot_a, double h, double inv_h)
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
// Candidate screens: queue every partner within the screening radius of an
// old or new position of a moved atom (and, for single-atom moves and flips,
// every atom of the molecule).  The candidates go in 64-candidate steps: lane
// l takes candidates base + l and base + 32 + l, so the warp's record loads
// are contiguous (no shared-memory bank conflicts).  A screening block is U
// steps (U = 4, and one block of 1 to 3 steps for the rest of the K
// candidates); the loads and arithmetic of its steps are issued before any
// queue store, and the queue is filled in ascending candidate order
// afterwards.  Only the last step of a block can reach past the K staged
// atoms; its lanes there read the first padding record (no molecule, never
// within reach), so no lane branches.  Entries past QW are counted but not
// stored.
// ---------------------------------------------------------------------------

// append the hits of one 64-candidate step (candidate c = base + lane for bit
// b0, c + 32 for b1) in ascending candidate order; lanes without a hit, and
// hits past QW, write the discard slot
__device__ __forceinline__ void queue_step2(const WarpScr &S, int lane, int &qlen, unsigned b0, unsigned b1, int c)
{
    const unsigned lt = (1u << lane) - 1u;
    const int n0 = __popc(b0);
    const int e0 = ((b0 >> lane) & 1u) ? min(qlen + __popc(b0 & lt), QW) : QW;
    const int e1 = ((b1 >> lane) & 1u) ? min(qlen + n0 + __popc(b1 & lt), QW) : QW;
    S.qc[e0] = c;
    S.qc[e1] = c + 32;
    qlen += n0 + __popc(b1);
}

// append the hits of one 32-candidate step (candidate c = base + lane)
__device__ __forceinline__ void queue_step(const WarpScr &S, int lane, int &qlen, unsigned b, int c)
{
    const unsigned lt = (1u << lane) - 1u;
    const int e = ((b >> lane) & 1u) ? min(qlen + __popc(b & lt), QW) : QW;
    S.qc[e] = c;
    qlen += __popc(b);
}

// The K candidates in screening blocks.  WHOLE (one-warp groups, where the
// smaller code measured faster): 4-step blocks only, every step clamped to
// K.  Otherwise 4 steps while more than 192 candidates remain (only the last
// step can reach past K), then one block of the 1 to 3 steps that cover the
// rest.
template <bool WHOLE, class Steps>
__device__ __forceinline__ int screen_blocks(int K, const Steps &st)
{
    int qlen = 0, base = 0;
    if constexpr (WHOLE) {
        for (; base < K; base += 64 * SCREEN_U) st.template run<SCREEN_U, true>(base, qlen);
    } else {
        for (; K - base > 64 * (SCREEN_U - 1); base += 64 * SCREEN_U) st.template run<SCREEN_U, false>(base, qlen);
        const int rem = (K - base + 63) >> 6;   // 0 to 3
        if (rem == 3) st.template run<3, false>(base, qlen);
        else if (rem == 2) st.template run<2, false>(base, qlen);
        else if (rem == 1) st.template run<1, false>(base, qlen);
    }
    return qlen;
}

// candidate pair of step u of a block: below K except in the block's last step
// (or in any step, CLAMP)
template <int U, bool CLAMP>
__device__ __forceinline__ void step_pair(const Group &G, int K, int base, int u, int lane, int4 &r0, int4 &r1)
{
    int c0 = base + 64 * u + lane, c1 = c0 + 32;
    if (CLAMP || u == U - 1) {
        c0 = min(c0, K);
        c1 = min(c1, K);
    }
    r0 = G.rec[c0];
    r1 = G.rec[c1];
}

// Atom translation from qo to qo + e: the old distance from the exact int32
// differences, the new one as r'^2 = r^2 - 2 d.e + |e|^2 (fixed-point units);
// the lane's two candidates in packed FP32 pairs.
struct AtomSteps {
    const Group &G;
    const WarpScr &S;
    int K, lane, wi;
    Q3 qo;
    f2_t mx, my, mz, e2;
    float r2q;
    template <int U, bool CLAMP>
    __device__ __forceinline__ void run(int base, int &qlen) const
    {
        unsigned b0[U], b1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int4 r0, r1;
            step_pair<U, CLAMP>(G, K, base, u, lane, r0, r1);
            const f2_t X = pk(dq((uint32_t)r0.x, qo.x), dq((uint32_t)r1.x, qo.x));
            const f2_t Y = pk(dq((uint32_t)r0.y, qo.y), dq((uint32_t)r1.y, qo.y));
            const f2_t Z = pk(dq((uint32_t)r0.z, qo.z), dq((uint32_t)r1.z, qo.z));
            const f2_t r2o = fma2(Z, Z, fma2(Y, Y, mul2(X, X)));
            const f2_t r2n = fma2(Z, mz, fma2(Y, my, fma2(X, mx, add2(r2o, e2))));
            float a0, a1, n0, n1;
            upk(r2o, a0, a1);
            upk(r2n, n0, n1);
            const bool p0 = ((fminf(a0, n0) < r2q) & (r0.w != PAD_W)) | ((r0.w ^ wi) < 16);
            const bool p1 = ((fminf(a1, n1) < r2q) & (r1.w != PAD_W)) | ((r1.w ^ wi) < 16);
            b0[u] = __ballot_sync(FULL, p0);
            b1[u] = __ballot_sync(FULL, p1);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) queue_step2(S, lane, qlen, b0[u], b1[u], base + 64 * u + lane);
    }
};

template <bool WHOLE>
__device__ __forceinline__ int screen_atom(const Group &G, const WarpScr &S, int K, int lane, const Q3 &qo,
                                           const Q3 &qn, int wi, float r2q)
{
    const float ex = dq(qn.x, qo.x), ey = dq(qn.y, qo.y), ez = dq(qn.z, qo.z);
    const float ee = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    const AtomSteps st{G, S, K, lane, wi, qo, pk(-2.f * ex, -2.f * ex), pk(-2.f * ey, -2.f * ey),
                       pk(-2.f * ez, -2.f * ez), pk(ee, ee), r2q};
    return screen_blocks<WHOLE>(K, st);
}

// Flip: distance of every candidate to the two atoms whose types swap.
struct FlipSteps {
    const Group &G;
    const WarpScr &S;
    int K, lane, wi;
    Q3 qp, qq;
    float r2q;
    template <int U, bool CLAMP>
    __device__ __forceinline__ void run(int base, int &qlen) const
    {
        unsigned b0[U], b1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int4 r0, r1;
            step_pair<U, CLAMP>(G, K, base, u, lane, r0, r1);
            f2_t X = pk(dq((uint32_t)r0.x, qp.x), dq((uint32_t)r1.x, qp.x));
            f2_t Y = pk(dq((uint32_t)r0.y, qp.y), dq((uint32_t)r1.y, qp.y));
            f2_t Z = pk(dq((uint32_t)r0.z, qp.z), dq((uint32_t)r1.z, qp.z));
            const f2_t rp = fma2(Z, Z, fma2(Y, Y, mul2(X, X)));
            X = pk(dq((uint32_t)r0.x, qq.x), dq((uint32_t)r1.x, qq.x));
            Y = pk(dq((uint32_t)r0.y, qq.y), dq((uint32_t)r1.y, qq.y));
            Z = pk(dq((uint32_t)r0.z, qq.z), dq((uint32_t)r1.z, qq.z));
            const f2_t rq = fma2(Z, Z, fma2(Y, Y, mul2(X, X)));
            float a0, a1, n0, n1;
            upk(rp, a0, a1);
            upk(rq, n0, n1);
            const bool p0 = ((fminf(a0, n0) < r2q) & (r0.w != PAD_W)) | ((r0.w ^ wi) < 16);
            const bool p1 = ((fminf(a1, n1) < r2q) & (r1.w != PAD_W)) | ((r1.w ^ wi) < 16);
            b0[u] = __ballot_sync(FULL, p0);
            b1[u] = __ballot_sync(FULL, p1);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) queue_step2(S, lane, qlen, b0[u], b1[u], base + 64 * u + lane);
    }
};

template <bool WHOLE>
__device__ __forceinline__ int screen_flip(const Group &G, const WarpScr &S, int K, int lane, const Q3 &qp,
                                           const Q3 &qq, int wi, float r2q)
{
    const FlipSteps st{G, S, K, lane, wi, qp, qq, r2q};
    return screen_blocks<WHOLE>(K, st);
}

// Rigid molecule move: the three atoms, old and new (molecule partners are
// not queued: their distances do not change).
__device__ __noinline__ int screen_mol(const Group G, const WarpScr S, int K, int lane, const Q3 *qo, const Q3 *qn,
                                       int wi, float r2q)
{
    int qlen = 0;
    for (int base = 0; base < K; base += 32) {
        const int c = base + lane;
        const int4 r = G.rec[c < K ? c : K];
        float mn = 3.0e38f;
        for (int s = 0; s < 3; ++s) mn = fminf(mn, fminf(r2_q(r, qo[s]), r2_q(r, qn[s])));
        const bool hit = (mn < r2q) && r.w != PAD_W && ((r.w ^ wi) >= 16);
        queue_step(S, lane, qlen, __ballot_sync(FULL, hit), c);
    }
    return qlen;
}

// ---------------------------------------------------------------------------
// FP32 interaction passes over the queue (each lane takes entries lane and
// lane + 32): partial (dE, mag, guard) per lane.  Distances come from the
// exact int32 differences of the raw records, converted once per axis (and
// scaled by h^2): at most about 7 units of 2^-24 relative error in r^2.
// ---------------------------------------------------------------------------
struct Acc32 {
    float dE, mag;
    int guard;
    int cnt;                    // pair-potential evaluations inside their range
};

__device__ __forceinline__ void add_wca(const ModelDev &md, float r2, int ab, float sign, Acc32 &a)
{
    if (r2 < md.rc2f[ab]) {
        float u, m;
        wca32(md, r2, ab, u, m);
        a.dE = fmaf(sign, u, a.dE);
        a.mag += m;
        a.cnt += 1;
    }
}

__device__ __forceinline__ void add_fene(const ModelDev &md, float r2, int ab, float sign, Acc32 &a)
{
    if (r2 * md.invR2f[ab] >= md.bond_guard_f) {
        a.guard = 1;
        return;
    }
    float u, m;
    fene32(md, r2, ab, u, m);
    a.dE = fmaf(sign, u, a.dE);
    a.mag += m;
    a.cnt += 1;
}

// Masked forms for the hot passes: every lane evaluates every term and
// multiplies it by 0 or 1, so the warp never diverges (in a latency-bound warp
// a divergent branch costs more than the arithmetic it skips).  Terms that are
// on add exactly what add_wca / add_fene add.
__device__ __forceinline__ void wca_m(const ModelDev &md, float r2, int ab, float sign, Acc32 &a)
{
    float u, m;
    wca32(md, r2, ab, u, m);
    const bool in = r2 < md.rc2f[ab];
    const float on = in ? 1.f : 0.f;
    a.dE = fmaf(sign * on, u, a.dE);
    a.mag = fmaf(on, m, a.mag);
    a.cnt += in;
}

__device__ __forceinline__ void fene_m(const ModelDev &md, float r2, int ab, float sign, bool bonded, Acc32 &a)
{
    const float x = r2 * md.invR2f[ab];
    const bool stretched = x >= md.bond_guard_f;
    a.guard |= (bonded && stretched) ? 1 : 0;
    const bool on = bonded && !stretched;
    const float xs = on ? x : 0.f;
    const float y = 1.0f - xs;
    const float l = __logf(y);
    const float f = on ? 1.f : 0.f;
    a.cnt += on;
    a.dE = fmaf(sign * f, md.nkef * l, a.dE);
    a.mag = fmaf(f, md.kef * (fabsf(l) + __fdividef(xs, y) + 1.0f), a.mag);
}

// squared distance in sigma units of queued record r to position q; a padding
// record is beyond every cutoff
__device__ __forceinline__ float cand_r2(const int4 &r, const Q3 &q, float h2)
{
    return r.w == PAD_W ? 1.0e30f : r2_q(r, q) * h2;
}

// Entry e of the queue, or the padding record K when e is past the queue or
// names one of the moved atoms.
__device__ __forceinline__ int queued(const WarpScr &S, int e, int nq, int K, int k0, int k1)
{
    const int cq = S.qc[e];   // e < QW: inside the queue array
    return (e < nq && cq != k0 && cq != k1) ? cq : K;
}

__device__ __forceinline__ Acc32 inter_atom(const Group &G, const WarpScr &S, int nq, int lane, const ModelDev &md,
                                            int K, int k, int wi, int ti, const Q3 &qo, const Q3 &qn, float h2)
{
    Acc32 a{0.f, 0.f, 0, 0};
    const int slots = nq > 32 ? 2 : 1;   // warp-uniform
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (s < slots) {
            const int4 r = G.rec[queued(S, lane + 32 * s, nq, K, k, k)];
            const int ab = 3 * ti + rec_type(r.w);
            const bool bonded = (r.w ^ wi) < 16;
            const float r2o = cand_r2(r, qo, h2), r2n = cand_r2(r, qn, h2);
            wca_m(md, r2o, ab, -1.f, a);
            wca_m(md, r2n, ab, 1.f, a);
            fene_m(md, r2o, ab, -1.f, bonded, a);
            fene_m(md, r2n, ab, 1.f, bonded, a);
        }
    }
    return a;
}

__device__ __forceinline__ Acc32 inter_flip(const Group &G, const WarpScr &S, int nq, int lane, const ModelDev &md,
                                            int K, int kp, int kq, int wi, int tp, int tq, const Q3 &qp,
                                            const Q3 &qq, float h2)
{
    Acc32 a{0.f, 0.f, 0, 0};
    const int slots = nq > 32 ? 2 : 1;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (s < slots) {
            const int4 r = G.rec[queued(S, lane + 32 * s, nq, K, kp, kq)];
            const int tj = rec_type(r.w);
            const bool bonded = (r.w ^ wi) < 16;
            const float rp = cand_r2(r, qp, h2), rq = cand_r2(r, qq, h2);
            // atom p: type tp -> tq; atom q: type tq -> tp
            wca_m(md, rp, 3 * tp + tj, -1.f, a);
            wca_m(md, rp, 3 * tq + tj, 1.f, a);
            wca_m(md, rq, 3 * tq + tj, -1.f, a);
            wca_m(md, rq, 3 * tp + tj, 1.f, a);
            fene_m(md, rp, 3 * tp + tj, -1.f, bonded, a);
            fene_m(md, rp, 3 * tq + tj, 1.f, bonded, a);
            fene_m(md, rq, 3 * tq + tj, -1.f, bonded, a);
            fene_m(md, rq, 3 * tp + tj, 1.f, bonded, a);
        }
    }
    return a;
}

__device__ __noinline__ Acc32 inter_mol(const Group G, const WarpScr S, int nq, int lane, const ModelDev &md, int K,
                                        const int *t3, const Q3 *qo, const Q3 *qn, float h2)
{
    Acc32 a{0.f, 0.f, 0, 0};
    for (int s = 0; s < 2; ++s) {
        const int4 r = G.rec[queued(S, lane + 32 * s, nq, K, -1, -1)];
        const int tj = rec_type(r.w);
        for (int m = 0; m < 3; ++m) {
            const int ab = 3 * t3[m] + tj;
            wca_m(md, cand_r2(r, qo[m], h2), ab, -1.f, a);
            wca_m(md, cand_r2(r, qn[m], h2), ab, 1.f, a);
        }
    }
    return a;
}

// intramolecular terms of a rotation (FP32, one lane), added to part
__device__ __noinline__ Acc32 rot_intra32(const ModelDev &md, const Q3 *qo, const Q3 *qn, const int *t3, float hf,
                                          Acc32 part)
{
    const int pk3[3] = {0, 0, 1}, pl3[3] = {1, 2, 2};
    for (int pr = 0; pr < 3; ++pr) {
        const int kk = pk3[pr], ll = pl3[pr];
        const int ab = 3 * t3[kk] + t3[ll];
        const int4 ro = make_int4((int)qo[ll].x, (int)qo[ll].y, (int)qo[ll].z, 0);
        const int4 rn = make_int4((int)qn[ll].x, (int)qn[ll].y, (int)qn[ll].z, 0);
        const float r2o = r2_int32f(ro, qo[kk], hf);
        const float r2n = r2_int32f(rn, qn[kk], hf);
        add_wca(md, r2o, ab, -1.f, part);
        add_wca(md, r2n, ab, 1.f, part);
        add_fene(md, r2o, ab, -1.f, part);
        add_fene(md, r2n, ab, 1.f, part);
    }
    return part;
}

// ---------------------------------------------------------------------------
// Everything one attempt needs that is the same for all attempts of the cell
// ---------------------------------------------------------------------------
struct CellCtx {
    const ModelDev *md;
    const MixDev *mx;
    RecView rv;
    int K, n, cellL, nc;
    uint32_t P[3];          // cell centre (fixed point): origin of the conflict test's frame
    uint32_t shift[3];
    double h, inv_h, T64;
    float hf, h2f;          // h and h^2 in FP32
    float pre_r2;           // screening radius squared (sigma units): 1.01 x the largest WCA cutoff squared
    float r2q;              // the same in fixed-point units squared (the screens' units)
    float gap, T32;
    int *err;
};

__device__ __forceinline__ PosH local_of(const CellCtx &c, const Q3 &q)
{
    return PosH{dq(q.x, c.P[0]), dq(q.y, c.P[1]), dq(q.z, c.P[2])};
}

// Evaluate attempt `jr` of the current chunk (one warp, state read-only) and
// return its outcome (the same in every lane); with W > 1 lane 0 also leaves
// in N what the conflict test of the later attempts of the round reads.
template <int PREC, int W>
__device__ Res evaluate(const CellCtx &cx, const Group &G, const WarpScr &S, Near *N, int jr, int lane)
{
    const ModelDev &md = *cx.md;
    // the attempt's draws, decoded by the cell-list build (site rank, move type,
    // flip axis, integer displacement or rotation words; threshold words)
    const uint32_t *w = G.rnd + 8 * jr;
    const uint4 dsc = *(const uint4 *)w;
    const int K = cx.K, n = cx.n;
    const int k = (int)(dsc.x & 0xFFFFu);
    const int mvt = (int)((dsc.x >> 16) & 3u);
    const int4 rk = G.rec[k];
    const int wi = rk.w;
    const int mol = rec_mol(wi);
    int status = MC_ST_EVALUATED;
    int flags = 0, accept = 0, inter = 0;
    float scale = 0.f, dE32 = 0.f;
    double dE64 = __longlong_as_double(0x7FF8000000000000ll);

    int ks[3] = {k, -1, -1};
    Q3 qo[3] = {}, qn[3] = {};
    int t3o[3] = {0, 0, 0}, t3n[3] = {0, 0, 0};
    int nmv = 1;
    if (mvt == MC_MOVE_ATOM) {
        qo[0] = Q3{(uint32_t)rk.x, (uint32_t)rk.y, (uint32_t)rk.z};
        qn[0] = Q3{qo[0].x + dsc.y, qo[0].y + dsc.z, qo[0].z + dsc.w};
        t3o[0] = t3n[0] = rec_type(wi);
        if (cell_local(qn[0].x, qn[0].y, qn[0].z, cx.shift, cx.nc) != cx.cellL) status = MC_ST_LEFT_CELL;
    } else {
        // the molecule's atoms in the own cell
        int k0 = -1, k1 = -1, k2 = -1;
        for (int j = 0; j < n; ++j) {
            const int wj = G.rec[j].w;
            if (rec_mol(wj) == mol) {
                const int sl = rec_slot(wj);
                if (sl == 0) k0 = j;
                if (sl == 1) k1 = j;
                if (sl == 2) k2 = j;
            }
        }
        if (mvt == MC_MOVE_FLIP) {
            const int axis = (int)((dsc.x >> 18) & 3u);
            const int kp = axis == 0 ? k1 : k0, kq = axis == 2 ? k1 : k2;
            if (kp < 0 || kq < 0) {
                status = MC_ST_NOT_IN_CELL;
            } else {
                nmv = 2;
                ks[0] = kp;
                ks[1] = kq;
                const int4 rp = G.rec[kp], rq = G.rec[kq];
                qo[0] = qn[0] = Q3{(uint32_t)rp.x, (uint32_t)rp.y, (uint32_t)rp.z};
                qo[1] = qn[1] = Q3{(uint32_t)rq.x, (uint32_t)rq.y, (uint32_t)rq.z};
                t3o[0] = rec_type(rp.w);
                t3o[1] = rec_type(rq.w);
                t3n[0] = t3o[1];
                t3n[1] = t3o[0];
            }
        } else {
            ks[0] = k0;
            ks[1] = k1;
            ks[2] = k2;
            if (k0 < 0 || k1 < 0 || k2 < 0) {
                status = MC_ST_NOT_IN_CELL;
            } else {
                nmv = 3;
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    const int4 rs = G.rec[ks[s]];
                    qo[s] = Q3{(uint32_t)rs.x, (uint32_t)rs.y, (uint32_t)rs.z};
                    t3o[s] = t3n[s] = rec_type(rs.w);
                }
                if (mvt == MC_MOVE_MOL_TRANS) {
#pragma unroll
                    for (int s = 0; s < 3; ++s) qn[s] = Q3{qo[s].x + dsc.y, qo[s].y + dsc.z, qo[s].z + dsc.w};
                } else {
                    uint32_t a9[9];
                    if (lane == 0) {
                        uint32_t qq[3][3], qr[3][3];
                        for (int s = 0; s < 3; ++s) {
                            qq[s][0] = qo[s].x;
                            qq[s][1] = qo[s].y;
                            qq[s][2] = qo[s].z;
                        }
                        rotate_molecule(qq, qr, w + 1, cx.mx->rot_a, cx.h, cx.inv_h);
                        for (int s = 0; s < 3; ++s)
                            for (int ax = 0; ax < 3; ++ax) a9[3 * s + ax] = qr[s][ax];
                    }
#pragma unroll
                    for (int i = 0; i < 9; ++i) a9[i] = __shfl_sync(FULL, a9[i], 0);
#pragma unroll
                    for (int s = 0; s < 3; ++s) qn[s] = Q3{a9[3 * s], a9[3 * s + 1], a9[3 * s + 2]};
                }
#pragma unroll
                for (int s = 0; s < 3; ++s)
                    if (cell_local(qn[s].x, qn[s].y, qn[s].z, cx.shift, cx.nc) != cx.cellL) status = MC_ST_LEFT_CELL;
            }
        }
    }

    // the FP64 ordered sum of this move and its decision (-1: bond break)
    auto exact = [&](double thr, int nq) {
        Move mv;
        mv.n = nmv;
        mv.mol = mol;
        mv.moves_pos = mvt != MC_MOVE_FLIP;
        mv.intra = mvt == MC_MOVE_MOL_ROT;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            mv.site[s] = s < nmv ? rec_site(G.rec[ks[s]].w) : -1;
            mv.to[s] = t3o[s];
            mv.tn[s] = t3n[s];
            mv.qo[s][0] = qo[s].x;
            mv.qo[s][1] = qo[s].y;
            mv.qo[s][2] = qo[s].z;
            mv.qn[s][0] = qn[s].x;
            mv.qn[s][1] = qn[s].y;
            mv.qn[s][2] = qn[s].z;
        }
        double e64 = 0.0;
        int cnt64 = 0;
        const int st = dE64_ordered(mv, cx.rv, S, K, nq, md, cx.h, cx.hf, cx.pre_r2, lane, cx.err, e64, cnt64);
        dE64 = e64;
        if (PREC == MC_PREC_FP64) inter = cnt64;
        return (st == MC_ST_EVALUATED) ? ((e64 <= thr) ? 1 : 0) : -1;
    };

    if (status == MC_ST_EVALUATED) {
        int qlen;
        if (mvt == MC_MOVE_ATOM) {
            qlen = screen_atom<W == 1>(G, S, K, lane, qo[0], qn[0], wi, cx.r2q);
        } else if (mvt == MC_MOVE_FLIP) {
            qlen = screen_flip<W == 1>(G, S, K, lane, qo[0], qo[1], wi, cx.r2q);
        } else {
            const Q3 a[3] = {qo[0], qo[1], qo[2]}, b[3] = {qn[0], qn[1], qn[2]};
            qlen = screen_mol(G, S, K, lane, a, b, wi, cx.r2q);
        }
        __syncwarp();
        const int nq = min(qlen, QW);
        const int nq64 = qlen <= QW ? qlen : -1;   // overflowed queue: the FP64 sum scans every atom
        if (PREC == MC_PREC_FP64) {
            const int dec = exact(G.thr64[jr], nq64);
            if (dec < 0) status = MC_ST_BOND_BREAK;
            accept = dec == 1;
        } else {
            const float thr32 = G.thr32[jr];
            Acc32 part;
            if (mvt == MC_MOVE_ATOM) {
                part = inter_atom(G, S, nq, lane, md, K, k, wi, t3o[0], qo[0], qn[0], cx.h2f);
            } else if (mvt == MC_MOVE_FLIP) {
                part = inter_flip(G, S, nq, lane, md, K, ks[0], ks[1], wi, t3o[0], t3o[1], qo[0], qo[1], cx.h2f);
            } else {
                const int tm[3] = {t3o[0], t3o[1], t3o[2]};
                const Q3 ro[3] = {qo[0], qo[1], qo[2]}, rn[3] = {qn[0], qn[1], qn[2]};
                part = inter_mol(G, S, nq, lane, md, K, tm, ro, rn, cx.h2f);
                if (mvt == MC_MOVE_MOL_ROT && lane == 0) part = rot_intra32(md, ro, rn, tm, cx.hf, part);
            }
            if (qlen > QW) part.guard = 1;
            inter = part.cnt;
            dE32 = warp_sum_f(part.dE);
            const float mag = warp_sum_f(part.mag);
            const int guard = __any_sync(FULL, part.guard);
            scale = mag;
            const float diff = fabsf(dE32 - thr32);
            const float marg = cx.gap * mag + 1e-6f * (cx.T32 + fabsf(thr32) + fabsf(dE32));
            if (guard || !(diff > marg)) {
                // retake in FP64: exact Delta E against the exact threshold
                flags = 1;
                __syncwarp();
                const unsigned long long u52 = ((unsigned long long)w[4] << 20) | (unsigned long long)(w[5] >> 12);
                const double u = __dmul_rn((double)(2ull * u52 + 1ull), 0x1p-53);
                const double thr = -__dmul_rn(cx.T64, ln_series(u));
                const int dec = exact(thr, nq64);
                if (dec < 0) status = MC_ST_BOND_BREAK;
                accept = dec == 1;
            } else {
                accept = dE32 <= thr32;
            }
        }
    }

    Res R;
    R.status = status;
    R.accept = accept;
    R.flags = flags;
    R.mvt = mvt;
    R.nmv = nmv;
    R.site = rec_site(wi);
    R.mol = mol;
    R.dE32 = dE32;
    R.scale = scale;
    R.dE64 = dE64;
    R.pairs = (mvt == MC_MOVE_MOL_TRANS || mvt == MC_MOVE_MOL_ROT) ? 6 : 2;
    R.inter = inter;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        R.ks[s] = ks[s];
        R.t3n[s] = t3n[s];
        R.qn[s][0] = qn[s].x;
        R.qn[s][1] = qn[s].y;
        R.qn[s][2] = qn[s].z;
    }
    if (W > 1 && lane == 0) {
        // positions the move reads or writes, for the conflict test of the commit
        int na = 0;
        if (status == MC_ST_EVALUATED) {
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                if (s < nmv) {
                    const PosH o = local_of(cx, qo[s]);
                    N->px[na] = o.x; N->py[na] = o.y; N->pz[na] = o.z; ++na;
                    if (mvt != MC_MOVE_FLIP) {
                        const PosH m = local_of(cx, qn[s]);
                        N->px[na] = m.x; N->py[na] = m.y; N->pz[na] = m.z; ++na;
                    }
                }
            }
        }
        N->accept = accept;
        N->mol = mol;
        N->nat = na;
    }
    return R;
}

// Could an earlier accepted attempt of the round have changed the evaluation
// of attempt wb?  Same molecule, or atoms within the conflict radius (1.01 x
// the largest cutoff, fixed-point units squared).  One warp: the lanes take
// the atom pairs of all earlier attempts at once (entries of attempts at or
// after wb are read but masked); every lane returns the same answer.
template <int W>
__device__ __forceinline__ bool clashes(const Near *near, int wb, float rconf, int lane)
{
    const Near &B = near[wb];
    bool hit = false;
#pragma unroll
    for (int wa = 0; wa < W - 1; ++wa) {
        const Near &A = near[wa];
        const bool live = (wa < wb) && A.accept != 0;
        hit |= live && A.mol == B.mol;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int p = min(lane + 32 * m, 35);         // atom pair (i, j); lanes past 35 repeat pair 35
            const int i = p / 6, j = p - 6 * (p / 6);
            const float dx = A.px[i] - B.px[j], dy = A.py[i] - B.py[j], dz = A.pz[i] - B.pz[j];
            hit |= live && i < A.nat && j < B.nat && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rconf;
        }
    }
    return __any_sync(FULL, hit);
}

// This lane's count of attempt R (see Tally).
__device__ __forceinline__ unsigned tally_inc(const Res &R, int lane)
{
    const bool evaluated = R.status == MC_ST_EVALUATED || R.status == MC_ST_BOND_BREAK;
    const bool geom = R.status == MC_ST_LEFT_CELL || R.status == MC_ST_NOT_IN_CELL;
    unsigned inc = lane == STAT_ATT + R.mvt;
    inc += (lane == STAT_ACC + R.mvt) & (R.accept != 0);
    inc += (lane == STAT_REJ_GEOM) & geom;
    inc += (lane == STAT_REJ_BOND) & (R.status == MC_ST_BOND_BREAK);
    inc += ((lane == STAT_PAIRS) & evaluated) ? (unsigned)R.pairs : 0u;
    inc += (lane == STAT_RECHECK) ? (unsigned)R.flags : 0u;
    return inc;
}

// Apply attempt R (number `at` in the cell) to the staged state and log it.
// One thread (lane 0 of the warp that evaluated it).  A moved atom whose
// fixed-point coordinate wraps around the box counts the periodic image it
// enters (img, per global site): only the cell that owns the atom moves it,
// so the counts need no atomics, and the per-commit wraps add up to those of
// the cell's net displacement.
template <int PREC>
__device__ __forceinline__ void commit(const Group &G, const Res &R, int at, const LogArgs &lg, const RepInfo &ri,
                                       uint64_t sweep, int own_start, int *img)
{
    if (R.accept) {
        if (R.mvt == MC_MOVE_FLIP) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                int4 rs = G.rec[R.ks[s]];
                rs.w = (rs.w & ~3) | R.t3n[s];
                G.rec[R.ks[s]] = rs;
            }
        } else {
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                if (s < R.nmv) {
                    const int ks = R.ks[s];
                    int4 rs = G.rec[ks];
                    const uint32_t o3[3] = {(uint32_t)rs.x, (uint32_t)rs.y, (uint32_t)rs.z};
                    int *im = img + 3 * (size_t)(ri.site_off + rec_site(rs.w));
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        const long long moved = (long long)o3[ax] + (long long)(int)(R.qn[s][ax] - o3[ax]);
                        if (moved < 0) im[ax] -= 1;
                        else if (moved >= 4294967296ll) im[ax] += 1;
                    }
                    rs.x = (int)R.qn[s][0];
                    rs.y = (int)R.qn[s][1];
                    rs.z = (int)R.qn[s][2];
                    G.rec[ks] = rs;
                }
            }
        }
    }
    if (lg.base != nullptr) {
        const uint64_t sl = sweep - lg.sweep0;
        mc_log_entry *e = lg.base + (size_t)ri.site_off * (size_t)lg.n_sweeps + (size_t)sl * (size_t)ri.n_sites +
                          (size_t)(own_start - ri.site_off) + (size_t)at;
        e->site = R.site;
        e->move = (int16_t)R.mvt;
        e->flags = (int16_t)R.flags;
        e->status = R.status;
        e->accepted = R.accept;
        const double dE_mode = PREC == MC_PREC_FP64 ? R.dE64 : (double)R.dE32;
        e->dE = R.status == MC_ST_EVALUATED ? dE_mode : __longlong_as_double(0x7FF8000000000000ll);
        e->dE64 = R.dE64;
        e->scale = (double)R.scale;
    }
}

// copy the model tables and move mix into the block's shared memory
__device__ __forceinline__ void load_tables(const DevState &d, ModelDev &md, MixDev &mx)
{
    const int *src = (const int *)d.model;
    int *dst = (int *)&md;
    for (int i = threadIdx.x; i < (int)(sizeof(ModelDev) / 4); i += blockDim.x) dst[i] = src[i];
    const int *src2 = (const int *)d.mix;
    int *dst2 = (int *)&mx;
    for (int i = threadIdx.x; i < (int)(sizeof(MixDev) / 4); i += blockDim.x) dst2[i] = src2[i];
}

// Once per launch, by the first thread of each group: the bulk-copy barrier
// and its phase parity (the caller synchronises the block afterwards).
__device__ __forceinline__ void init_group(unsigned char *gsmem, const DevState &d, int W)
{
    if (threadIdx.x % (32 * W) == 0) {
        const Group G = carve(gsmem, W);
        mbar_init(G.mbar);
        G.misc[MS_PHASE] = 0;
    }
}

// Ordering inside one persistent launch, cell by cell: a cell may start its
// phase of sweep s once every neighbour of a smaller colour has finished its
// phase (the neighbours' writes are then visible, and none of them still reads
// this cell's atoms; neighbours of a larger colour wait for this cell in turn).
// done[c] counts what cell c completed in the launch.  One-warp groups: its
// colour phases (s + 1 after sweep s), the cell list being complete at a grid
// barrier.  Multi-warp groups: its order passes too, two per sweep (2s + 1 once
// it is ordered in sweep s, 2s + 2 after its phase), and a phase also waits
// for every cell of its neighbourhood, itself included, to be ordered (no grid
// barrier between the order pass and the colours; measured faster for these
// schedules and slower for one-warp groups).  In run_cell, dep = s + 1 (0:
// ordered by kernel boundaries); wait_done waits for done[c] >= a count.
__device__ __forceinline__ void wait_done(const unsigned int *done, unsigned dep, int *err, unsigned limit)
{
    const unsigned lim = limit ? limit : (1u << 21);
    unsigned spins = 0;
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(done) : "memory");
        if (v >= dep) return;
        ++spins;
        // bounded; and once any wait of the launch has given up, the others stop too
        if ((spins & 4095u) == 0 && (*(volatile int *)err & ERR_TIMEOUT)) return;
        if (spins > lim) {
            atomicOr(err, ERR_TIMEOUT);
            return;
        }
    }
}

// The group's writes to the cell are complete (the caller synchronised the
// group): publish them and count the phase.  One thread.
__device__ __forceinline__ void signal_done(unsigned int *done)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(done) : "memory");
}

// All n attempts of active cell g of the colour, by the 32 W threads of one
// group (group index gid within the block, its shared memory at gsmem).
template <int PREC, int W>
__device__ void run_cell(const DevState &d, int buf, int colour, const LogArgs &lg, int g, const ModelDev &md,
                         const MixDev &mx, unsigned char *gsmem, int gid, unsigned dep)
{
    constexpr int T = 32 * W;          // threads per cell
    const int gt = threadIdx.x % T;
    const int lane = threadIdx.x & 31;
    const int wig = gt >> 5;
    const int cap = d.stencil_cap;
    const Group G = carve(gsmem, W);
    const WarpScr S = warp_scr(G, wig);

    // ---- which cell ----
    const int2 sl = d.act_slot ? d.act_slot[g] : make_int2(0, g);
    const int r = sl.x;
    const RepInfo ri = d.rep[r];
    const RepParam dy = d.par[r];
    const RepCtr ct = d.ctr[r];
    const int nc = ri.nc, h2 = nc >> 1;
    const int a_loc = sl.y;
    const int cx = 2 * (a_loc % h2) + (colour & 1);
    const int cy = 2 * ((a_loc / h2) % h2) + ((colour >> 1) & 1);
    const int cz = 2 * (a_loc / (h2 * h2)) + ((colour >> 2) & 1);
    const int cellL = (cz * nc + cy) * nc + cx;
    const int cellG = ri.cell_off + cellL;
    const bool raw = nc == 2;
    const int ns = raw ? 8 : 27;

    // ---- neighbourhood: own cell first.  The extents of the cells and the
    // random words of the first 32 attempts are loaded before waiting for the
    // neighbours (both are fixed for the sweep); the records only after ----
    uint4 rb0 = make_uint4(0, 0, 0, 0), rb1 = rb0;   // warp 0: attempt `lane`'s draws
    double th64 = 0.0;
    float th32 = 0.f;
    if (wig == 0) {
        int cnt = 0, cst = 0, wait_c = -1;
        unsigned wait_n = 0;
        if (lane < ns) {
            int ox, oy, oz;
            if (raw) {
                ox = lane & 1; oy = (lane >> 1) & 1; oz = lane >> 2;
            } else {
                const int kk = (lane == 0) ? 13 : (lane <= 13 ? lane - 1 : lane);   // 13 = (0,0,0)
                ox = kk % 3 - 1; oy = (kk / 3) % 3 - 1; oz = kk / 9 - 1;
            }
            const int nx = (cx + ox + nc) % nc, ny = (cy + oy + nc) % nc, nz = (cz + oz + nc) % nc;
            const int c = ri.cell_off + (nz * nc + ny) * nc + nx;
            const int ncol = (nx & 1) | ((ny & 1) << 1) | ((nz & 1) << 2);
            if (W == 1) {
                if (dep != 0 && ncol < colour) wait_c = c;
                wait_n = dep;
            } else {
                if (dep != 0) wait_c = c;
                wait_n = ncol < colour ? 2u * dep : 2u * dep - 1u;
            }
            cst = d.cell_start[c];
            cnt = d.cell_start[c + 1] - cst;
        }
        {
            const int n0 = __shfl_sync(FULL, cnt, 0), s0 = __shfl_sync(FULL, cst, 0);
            if (lane < n0) {
                const size_t slot = (size_t)s0 + (size_t)lane;
                rb0 = d.att_rnd[2 * slot];
                rb1 = d.att_rnd[2 * slot + 1];
                if (PREC == MC_PREC_FP64) th64 = d.att_thr64[slot];
                else th32 = d.att_thr32[slot];
            }
        }
        // one-warp groups wait before the offsets, multi-warp groups after
        // (each order measured faster for its schedule)
        if (W == 1 && wait_c >= 0) wait_done(d.cell_done + wait_c, wait_n, d.err, d.wait_limit);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane < ns) {
            G.cstart[lane] = cst;
            G.coff[lane] = incl - cnt;
        }
        if (lane == 31) {
            G.coff[ns] = incl;
            G.misc[MS_K] = incl;
        }
        if (lane == 0) {
            G.misc[MS_N] = cnt;
            G.misc[MS_START] = cst;
            G.misc[MS_FAIL] = 0;
        }
        if (W > 1 && wait_c >= 0) wait_done(d.cell_done + wait_c, wait_n, d.err, d.wait_limit);
        __syncwarp();
        if constexpr (W == 1) {
            // one-warp groups stage by bulk copies, one per cell, all
            // completing on the group's barrier (only when they fit)
            const int Kw = __shfl_sync(FULL, incl, 31);
            if (Kw + PADS <= cap) {
                if (lane == 0) mbar_arrive_expect(G.mbar, 16u * (unsigned)Kw);
                __syncwarp();
                if (lane < ns && cnt > 0)
                    bulk_to_smem(G.rec + (incl - cnt), d.rec[buf] + cst, 16u * (unsigned)cnt, G.mbar);
            }
        }
    }
    gsync<W>(gid);
    const int K = G.misc[MS_K];
    const int n = G.misc[MS_N];
    const int own_start = G.misc[MS_START];
    if (K + PADS > cap) {   // the neighbourhood does not fit: nothing is staged
        if (gt == 0) {
            atomicOr(d.err, ERR_STENCIL);
            d.cell_dE[cellG] = 0.0;
            if (dep != 0) signal_done(d.cell_done + cellG);
        }
        return;
    }

    if constexpr (W == 1) {
        // ---- stage (one warp): wait for the bulk copies (bounded), store the
        // first 32 attempts' draws; padding records
        // follow the K atoms (no molecule, never within reach: the screens and
        // the interaction passes read them instead of branching) ----
        const unsigned parity = (unsigned)G.misc[MS_PHASE];
        unsigned spins = 0;
        bool ok = true;
        while (!mbar_done(G.mbar, parity)) {
            if (++spins > (1u << 22)) {
                ok = false;
                break;
            }
        }
        if (!ok) G.misc[MS_FAIL] = 1;
        if (lane < n) {
            uint4 *wv = (uint4 *)(G.rnd + 8 * lane);
            wv[0] = rb0;
            wv[1] = rb1;
            if (PREC == MC_PREC_FP64) G.thr64[lane] = th64;
            else G.thr32[lane] = th32;
        }
        if (lane < PADS) G.rec[K + lane] = make_int4(0, 0, 0, PAD_W);
        __syncwarp();
        if (G.misc[MS_FAIL]) {
            // copies that never completed: record it, give them one more bounded
            // wait, and leave the cell untouched
            if (lane == 0) atomicOr(d.err, ERR_TIMEOUT);
            for (unsigned t2 = 0; t2 < (1u << 22) && !mbar_done(G.mbar, parity); ++t2) {
            }
            if (lane == 0 && dep != 0) signal_done(d.cell_done + cellG);
            return;
        }
        if (lane == 0) G.misc[MS_PHASE] = (int)(parity ^ 1u);   // the warp has read the parity
    } else {
        // ---- stage (W >= 2 warps): the raw records of the neighbourhood,
        // loaded straight from L2 (the waits above acquired the neighbours'
        // writes; .cg loads bypass L1, which may hold lines of an earlier
        // phase).  Lane j of every warp takes cell j, warp w its records w,
        // w + W, ..., several loads in flight.  Warp 0 stores the first 32
        // attempts' draws; padding records
        // follow the K atoms ----
        if (lane < ns) {
            const int off = G.coff[lane], cnt = G.coff[lane + 1] - off;
            const int4 *src = d.rec[buf] + G.cstart[lane];
            constexpr int su = W == 2 ? 8 : (W == 4 ? 4 : SU);   // a cell's records in one round trip
            for (int k0 = wig; k0 < cnt; k0 += su * W) {
                int4 v[su];
#pragma unroll
                for (int u = 0; u < su; ++u)
                    if (k0 + u * W < cnt) v[u] = __ldcg(src + k0 + u * W);
#pragma unroll
                for (int u = 0; u < su; ++u) {
                    const int k = k0 + u * W;
                    if (k < cnt) G.rec[off + k] = v[u];
                }
            }
        }
        if (wig == 0 && lane < n) {
            uint4 *wv = (uint4 *)(G.rnd + 8 * lane);
            wv[0] = rb0;
            wv[1] = rb1;
            if (PREC == MC_PREC_FP64) G.thr64[lane] = th64;
            else G.thr32[lane] = th32;
        }
        if (gt < PADS) G.rec[K + gt] = make_int4(0, 0, 0, PAD_W);
        gsync<W>(gid);
    }

    CellCtx c;
    c.md = &md;
    c.mx = &mx;
    c.K = K;
    c.n = n;
    c.cellL = cellL;
    c.nc = nc;
    c.shift[0] = ct.shift[0];
    c.shift[1] = ct.shift[1];
    c.shift[2] = ct.shift[2];
    // origin of the conflict test's frame: any point near the cell will do (the
    // test compares differences with a 1% margin); own atom 0 as staged
    const int4 p0 = n > 0 ? G.rec[0] : make_int4(0, 0, 0, 0);
    c.P[0] = (uint32_t)p0.x;
    c.P[1] = (uint32_t)p0.y;
    c.P[2] = (uint32_t)p0.z;
    c.h = ri.h;
    c.inv_h = ri.inv_h;
    c.hf = ri.hf;
    c.h2f = ri.h2f;
    c.T64 = dy.T;
    c.T32 = dy.T32;
    c.gap = md.recheck_gap_f;
    c.err = d.err;
    c.pre_r2 = ri.pre_r2;
    c.r2q = ri.r2q;
    const float rconf = ri.rconf;   // (1.01 rc)^2, fixed-point units
    c.rv.smem = G.rec;

    unsigned cnt = 0;                  // this lane's counter of the warp's tally
    unsigned inter_lane = 0;           // this lane's share of the committed attempts' in-range evaluations
    // the running energy: FP64 sums in FP64 mode; in FP32 mode the few
    // accepted Delta E of a cell are summed in FP32 (they carry FP32 errors
    // already) and the cell total joins the FP64 sum (every lane the same)
    float dEf = 0.f;
    double dE = 0.0;
    for (int a0 = 0; a0 < n; a0 += 32) {
        if (a0 > 0) {
            // random words and thresholds of the next chunk (cells with more than 32 atoms)
            if (wig == 0) {
                const int a = a0 + lane;
                if (a < n) {
                    const size_t slot = (size_t)own_start + (size_t)a;
                    uint4 *wv = (uint4 *)(G.rnd + 8 * lane);
                    wv[0] = d.att_rnd[2 * slot];
                    wv[1] = d.att_rnd[2 * slot + 1];
                    if (PREC == MC_PREC_FP64) G.thr64[lane] = d.att_thr64[slot];
                    else G.thr32[lane] = d.att_thr32[slot];
                }
            }
            gsync<W>(gid);
        }
        const int a_end = min(n, a0 + 32);
        int a = a0;
        while (a < a_end) {
            // evaluate attempts a .. a+nw-1, one per warp, on the same state
            const int nw = min(W, a_end - a);
            Res R;
            if (wig < nw) R = evaluate<PREC, W>(c, G, S, G.near + wig, a + wig - a0, lane);
            int adv = 1;
            if constexpr (W > 1) {
                gsync<W>(gid);
                // commit in order up to the first attempt an earlier accepted one may
                // have changed; when no attempt but possibly the last was accepted,
                // nothing can have changed (every warp reads the same flags)
                bool any_acc = false;
#pragma unroll
                for (int wa = 0; wa < W - 1; ++wa) any_acc |= (wa < nw - 1) && G.near[wa].accept != 0;
                adv = nw;
                if (any_acc) {
                    if (wig < nw) {
                        const bool cl = clashes<W>(G.near, wig, rconf, lane);
                        if (lane == 0) G.misc[MS_CLASH + wig] = cl;
                    }
                    gsync<W>(gid);
                    for (int j = 1; j < nw; ++j)
                        if (G.misc[MS_CLASH + j]) {
                            adv = j;
                            break;
                        }
                }
            } else {
                __syncwarp();
            }
            // committed attempts touch different molecules: each warp applies its own
            if (wig < adv) {
                if (lane == 0) commit<PREC>(G, R, a + wig, lg, ri, ct.sweep, own_start, d.img);
                cnt += tally_inc(R, lane);
                inter_lane += (unsigned)R.inter;
                if (R.accept) {
                    if (PREC == MC_PREC_FP64) dE = __dadd_rn(dE, R.dE64);
                    else dEf += R.flags ? (float)R.dE64 : R.dE32;
                }
            }
            if constexpr (W > 1) gsync<W>(gid);
            else __syncwarp();
            a += adv;
        }
    }

    // ---- write back the cell and publish it to the neighbours waiting for
    // it; then the counts, which nobody waits for: the warps' tallies in warp
    // order (one-warp groups reduce their lanes' counts before publishing,
    // multi-warp groups after: each order measured faster for its schedule) ----
    int4 *dst = d.rec[buf] + own_start;
    for (int kk = gt; kk < n; kk += T) dst[kk] = G.rec[kk];
    if constexpr (W == 1) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) inter_lane += __shfl_xor_sync(FULL, inter_lane, o);
    }
    gsync<W>(gid);   // every write-back is done
    if (gt == 0 && dep != 0) signal_done(d.cell_done + cellG);
    if constexpr (W > 1) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) inter_lane += __shfl_xor_sync(FULL, inter_lane, o);
        Tally &u = G.tally[wig];
        if (lane < TALLY_N) u.cnt[lane] = cnt;
        if (lane == 0) {
            u.inter = inter_lane;
            u.dEf = dEf;
            u.dE = dE;
        }
        gsync<W>(gid);   // every tally is written
    }
    if (wig == 0) {
        if constexpr (W > 1) {
            for (int j = 1; j < W; ++j) {
                const Tally &u = G.tally[j];
                if (lane < TALLY_N) cnt += u.cnt[lane];
                inter_lane += u.inter;
                if (PREC == MC_PREC_FP64) dE = __dadd_rn(dE, u.dE);
                else dEf += u.dEf;
            }
        }
        unsigned long long *st = d.stats + (size_t)r * STAT_N;
        const unsigned long long v =
            lane == STAT_PAIRS ? (unsigned long long)cnt * (unsigned long long)K : (unsigned long long)cnt;
        if (lane < TALLY_N && v != 0) atomicAdd(st + lane, v);
        if (lane == 0) {
            if (inter_lane) atomicAdd(st + STAT_INTER, (unsigned long long)inter_lane);
            d.cell_dE[cellG] = PREC == MC_PREC_FP64 ? dE : (double)dEf;
        }
    }
}

// threads per block of the phase kernel: one-warp groups get a block each, so
// that a warp that finishes its cell frees its place at once (with four cells
// per block the block held its place until its slowest cell was done)
template <int W>
__host__ __device__ constexpr int phase_threads() { return W == 1 ? 32 : block_threads<W>(); }

// One colour phase, one launch: group g of the grid owns active cell g.
// W = 1 serves large grids (many cells per SM): registers for fifteen resident blocks (128 per thread)
template <int PREC, int W>
__global__ void __launch_bounds__(phase_threads<W>(), W == 1 ? 15 : 1) phase_kernel(DevState d, int buf, int colour,
                                                                                 LogArgs lg)
{
    constexpr int CPB = phase_threads<W>() / (32 * W);
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ModelDev md;
    __shared__ MixDev mx;
    const int gid = threadIdx.x / (32 * W);
    unsigned char *gsmem = smem + (size_t)gid * group_bytes(d.stencil_cap, W);
    init_group(gsmem, d, W);
    load_tables(d, md, mx);
    __syncthreads();
    const int g = blockIdx.x * CPB + gid;
    if (g >= d.n_act) return;          // whole group leaves together
    run_cell<PREC, W>(d, buf, colour, lg, g, md, mx, gsmem, gid, 0u);
}

// Per replica (one block of at least BLOCK threads): add the sweep's accepted
// Delta E, the cells summed in a fixed partition over BLOCK lanes and a fixed
// reduction tree, whatever the block size, so the result is reproducible and
// the same for every schedule; count the sweep; advance the sweep counter.
__device__ void finalize_replica(const DevState &d, int r, double *red)
{
    const RepInfo ri = d.rep[r];
    const int ncell = ri.nc * ri.nc * ri.nc;
    if (threadIdx.x < BLOCK) {
        double s = 0.0;
        for (int c = threadIdx.x; c < ncell; c += BLOCK) s = __dadd_rn(s, d.cell_dE[ri.cell_off + c]);
        red[threadIdx.x] = s;
    }
    __syncthreads();
    for (int w = BLOCK / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        d.e_run[r] = __dadd_rn(d.e_run[r], red[0]);
        d.stats[(size_t)r * STAT_N + STAT_SWEEPS] += 1;
        d.ctr[r].sweep += 1;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(BLOCK) finalize_kernel(DevState d)
{
    __shared__ double red[BLOCK];
    finalize_replica(d, blockIdx.x, red);
}

// ---------------------------------------------------------------------------
// Persistent sweeps: one cooperative launch runs n_sweeps whole sweeps (cell
// list, 8 colour phases, finalisation).  The cell-list stages are separated
// by grid-wide barriers; the colour phases are ordered cell by cell
// (run_cell); the finalisation of sweep s shares a stage with the count of
// sweep s + 1, into the second count buffer, so a sweep takes 6 barriers.
// Every wait is bounded: after a few seconds it records ERR_TIMEOUT and the
// kernel leaves, instead of waiting forever.
// ---------------------------------------------------------------------------
struct GridBar {
    unsigned int *count;  // arrivals since the launch began (zero at launch)
    int *scan_tot;        // one per block: cell-count total of the block's chunk
};

// Arrive, then wait until every block has arrived as often as this one.  The
// count only grows, so no reset is needed between barriers; `target` is the
// caller's running total (thread 0 only).  The arrival is a release at gpu
// scope (it publishes every write the block made before the __syncthreads
// above it) and the polls are acquires (the block's reads after the
// __syncthreads below see every other block's published writes).  The wait is
// bounded.
__device__ bool grid_sync(const GridBar &gb, unsigned int &target, int *err, unsigned limit)
{
    const unsigned long long lim = limit ? limit : (1ull << 23);
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        target += gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(gb.count) : "memory");
        unsigned long long spins = 0;
        for (;;) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(gb.count) : "memory");
            if ((int)(v - target) >= 0) break;
            ++spins;
            if ((spins & 4095u) == 0 && (*(volatile int *)err & ERR_TIMEOUT)) {
                ok = 0;
                break;
            }
            if (spins > lim) {
                atomicOr(err, ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

// exclusive prefix sum over a block of NT threads (one value per thread)
template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int *tmp, int &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    int before = 0;
    total = 0;
    for (int w = 0; w < NT / 32; ++w) {
        if (w < warp) before += tmp[w];
        total += tmp[w];
    }
    __syncthreads();
    return before + x - v;
}

template <int PREC, int W>
__global__ void __launch_bounds__(block_threads<W>(), W == 1 ? 3 : 1) sweep_persistent(DevState d, int buf0,
                                                                                     int n_sweeps, GridBar gb)
{
    constexpr int T = 32 * W;
    constexpr int NT = block_threads<W>();
    constexpr int CPB = NT / T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ModelDev md;
    __shared__ MixDev mx;
    __shared__ double red[BLOCK];
    __shared__ int tmp[NT / 32];
    const int gid = threadIdx.x / T;
    unsigned char *gsmem = smem + (size_t)gid * group_bytes(d.stencil_cap, W);
    init_group(gsmem, d, W);
    load_tables(d, md, mx);
    __syncthreads();
    const int nthr = gridDim.x * NT;
    const int tid = blockIdx.x * NT + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const LogArgs none{nullptr, 0, 0};
    const int nC = d.n_cells;
    const int chunk = (nC + gridDim.x - 1) / gridDim.x;
    const int lo = min(nC, (int)blockIdx.x * chunk), hi = min(nC, lo + chunk);
    int buf = buf0;
    unsigned int bar_target = 0;
    // Every replica of a handle has done the same number of sweeps, so one
    // base serves all; it is read before any block can reach a finalisation.
    // Sweep s counts into cell_count for even s, cell_count2 for odd s.
    __shared__ uint64_t sweep0;
    if (threadIdx.x == 0) sweep0 = d.ctr[0].sweep;
    __syncthreads();
    // ---- cell list of the first sweep: count (cell_count is zero on entry) ----
    if (n_sweeps > 0)
        for (int g = tid; g < d.n_sites; g += nthr) cl_count_item(d, buf, g, sweep0, d.cell_count);
    for (int s = 0; s < n_sweeps; ++s) {
        int *const cnt = (s & 1) ? d.cell_count2 : d.cell_count;
        if (!grid_sync(gb, bar_target, d.err, d.wait_limit)) return;
        // ---- exclusive scan.  Small grids (at most 64 counts per thread): every
        // block sums the counts before its chunk and all of them itself, with no
        // grid-wide barrier.  Otherwise chunk totals first, then each block scans
        // its chunk ----
        const bool one_stage = nC <= 64 * NT;
        if (!one_stage) {
            int sum = 0;
            for (int c = lo + threadIdx.x; c < hi; c += NT) sum += cnt[c];
            int total;
            block_excl_scan<NT>(sum, tmp, total);
            if (threadIdx.x == 0) gb.scan_tot[blockIdx.x] = total;
            if (!grid_sync(gb, bar_target, d.err, d.wait_limit)) return;
        }
        {
            int off = 0, all = 0;
            if (one_stage) {
                for (int c = threadIdx.x; c < nC; c += NT) {
                    const int v = cnt[c];
                    all += v;
                    if (c < lo) off += v;
                }
            } else {
                for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) {
                    const int v = gb.scan_tot[b];
                    all += v;
                    if (b < (int)blockIdx.x) off += v;
                }
            }
            int t1, t2;
            block_excl_scan<NT>(off, tmp, t1);
            block_excl_scan<NT>(all, tmp, t2);
            int carry = t1;                       // sum of the totals of earlier blocks
            for (int base = lo; base < hi; base += NT) {
                const int c = base + threadIdx.x;
                const int v = c < hi ? cnt[c] : 0;
                int tile;
                const int ex = block_excl_scan<NT>(v, tmp, tile);
                if (c < hi) d.cell_start[c] = carry + ex;
                carry += tile;
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) d.cell_start[nC] = t2;
        }
        if (!grid_sync(gb, bar_target, d.err, d.wait_limit)) return;
        // ---- scatter (and clear the counts the next sweep will use, last read
        // by the previous sweep's scan), then order each cell and draw its
        // attempts' random numbers ----
        for (int g = tid; g < d.n_sites; g += nthr) cl_scatter_item(d, buf, buf ^ 1, g);
        for (int c = tid; c < nC; c += nthr) ((s & 1) ? d.cell_count : d.cell_count2)[c] = 0;
        if (!grid_sync(gb, bar_target, d.err, d.wait_limit)) return;
        if constexpr (W == 1) {
            // (one cell per warp: measured faster than four at a time in this
            // variant of the kernel, at 64000 molecules)
            for (int c = blockIdx.x * (NT / 32) + warp; c < nC; c += gridDim.x * (NT / 32))
                cl_order_cell(d, buf ^ 1, c, lane);
            if (!grid_sync(gb, bar_target, d.err, d.wait_limit)) return;
        } else {
            // (each ordered cell is published in cell_done: no grid-wide
            // barrier before the colours)
            for (int c = 4 * (blockIdx.x * (NT / 32) + warp); c < nC; c += 4 * gridDim.x * (NT / 32)) {
                cl_order_cells4(d, buf ^ 1, c, lane);
                __syncwarp();
                if (lane < 4 && c + lane < nC) signal_done(d.cell_done + c + lane);
            }
        }
        // ---- the 8 colours, ordered cell by cell (no grid-wide barrier between
        // colours: each cell waits for its neighbours of smaller colours) ----
        for (int colour = 0; colour < 8; ++colour)
            for (int g = blockIdx.x * CPB + gid; g < d.n_act; g += gridDim.x * CPB)
                run_cell<PREC, W>(d, buf ^ 1, colour, none, g, md, mx, gsmem, gid, (unsigned)s + 1u);
        if (!grid_sync(gb, bar_target, d.err, d.wait_limit)) return;
        // ---- finalise the sweep and, in the same stage, count the next
        // sweep's cell list (it reads only the positions written back above,
        // and the shift of sweep s + 1; the finalisation does not touch the
        // cell list) ----
        for (int r = blockIdx.x; r < d.n_rep; r += gridDim.x) finalize_replica(d, r, red);
        buf ^= 1;
        if (s + 1 < n_sweeps)
            for (int g = tid; g < d.n_sites; g += nthr)
                cl_count_item(d, buf, g, sweep0 + (uint64_t)s + 1u, (s & 1) ? d.cell_count : d.cell_count2);
    }
}

int sweep_binary_version()
{
    cudaFuncAttributes a{};
    if (cudaFuncGetAttributes(&a, finalize_kernel) != cudaSuccess) return -1;
    return a.binaryVersion;
}

size_t phase_smem_bytes(int stencil_cap, int warps_per_cell)
{
    const int nt = warps_per_cell > 4 ? 32 * warps_per_cell : BLOCK;
    return group_bytes(stencil_cap, warps_per_cell) * (size_t)(nt / (32 * warps_per_cell));
}

template <class K>
static bool set_kernel_smem(K kernel, int bytes)
{
    // one shared-memory carveout for every kernel of a sweep, so that the SMs
    // are not reconfigured between the cell-list kernels and the phases
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
}

int phase_set_smem_limit(int bytes_needed)
{
    // the attribute is per kernel, shared by all handles: keep the largest request
    static int granted = 0;
    const int bytes = std::max(granted, bytes_needed);
    granted = bytes;
    bool ok = true;
    ok &= set_kernel_smem(phase_kernel<MC_PREC_FP64, 1>, bytes);
    ok &= set_kernel_smem(phase_kernel<MC_PREC_FP64, 2>, bytes);
    ok &= set_kernel_smem(phase_kernel<MC_PREC_FP64, 4>, bytes);
    ok &= set_kernel_smem(phase_kernel<MC_PREC_FP64, 8>, bytes);
    ok &= set_kernel_smem(phase_kernel<MC_PREC_FP32, 1>, bytes);
    ok &= set_kernel_smem(phase_kernel<MC_PREC_FP32, 2>, bytes);
    ok &= set_kernel_smem(phase_kernel<MC_PREC_FP32, 4>, bytes);
    ok &= set_kernel_smem(phase_kernel<MC_PREC_FP32, 8>, bytes);
    ok &= set_kernel_smem(sweep_persistent<MC_PREC_FP64, 1>, bytes);
    ok &= set_kernel_smem(sweep_persistent<MC_PREC_FP64, 2>, bytes);
    ok &= set_kernel_smem(sweep_persistent<MC_PREC_FP64, 4>, bytes);
    ok &= set_kernel_smem(sweep_persistent<MC_PREC_FP64, 8>, bytes);
    ok &= set_kernel_smem(sweep_persistent<MC_PREC_FP32, 1>, bytes);
    ok &= set_kernel_smem(sweep_persistent<MC_PREC_FP32, 2>, bytes);
    ok &= set_kernel_smem(sweep_persistent<MC_PREC_FP32, 4>, bytes);
    ok &= set_kernel_smem(sweep_persistent<MC_PREC_FP32, 8>, bytes);
    const int full = cudaSharedmemCarveoutMaxShared;
    cudaFuncSetAttribute(finalize_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, full);
    cudaFuncSetAttribute(cl_count_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, full);
    cudaFuncSetAttribute(cl_scan_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, full);
    cudaFuncSetAttribute(cl_scatter_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, full);
    cudaFuncSetAttribute(cl_order_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, full);
    return ok ? 0 : -1;
}

template <int PREC>
static void launch_prec(const DevState &d, int buf, int W, const LogArgs &lg, cudaStream_t st)
{
    const int nt = W == 8 ? phase_threads<8>() : W == 4 ? phase_threads<4>() : W == 2 ? phase_threads<2>()
                                                                                  : phase_threads<1>();
    const int cpb = nt / (32 * W);
    const int blocks = (d.n_act + cpb - 1) / cpb;
    const size_t sm = group_bytes(d.stencil_cap, W) * (size_t)cpb;
    for (int colour = 0; colour < 8; ++colour) {
        if (W == 8) phase_kernel<PREC, 8><<<blocks, nt, sm, st>>>(d, buf, colour, lg);
        else if (W == 4) phase_kernel<PREC, 4><<<blocks, nt, sm, st>>>(d, buf, colour, lg);
        else if (W == 2) phase_kernel<PREC, 2><<<blocks, nt, sm, st>>>(d, buf, colour, lg);
        else phase_kernel<PREC, 1><<<blocks, nt, sm, st>>>(d, buf, colour, lg);
    }
}

void launch_colour_phases(const DevState &d, int buf, int warps_per_cell, const LogArgs &lg, cudaStream_t st)
{
    if (d.precision == MC_PREC_FP64) launch_prec<MC_PREC_FP64>(d, buf, warps_per_cell, lg, st);
    else launch_prec<MC_PREC_FP32>(d, buf, warps_per_cell, lg, st);
}

void launch_finalize(const DevState &d, cudaStream_t st)
{
    finalize_kernel<<<d.n_rep, BLOCK, 0, st>>>(d);
}

void launch_phases(const DevState &d, int buf, int warps_per_cell, const LogArgs &lg, cudaStream_t st)
{
    launch_colour_phases(d, buf, warps_per_cell, lg, st);
    launch_finalize(d, st);
}

template <int PREC, int W>
static void *persistent_fn()
{
    return (void *)sweep_persistent<PREC, W>;
}

static void *persistent_kernel(int prec, int W)
{
    if (prec == MC_PREC_FP64)
        return W == 8 ? persistent_fn<MC_PREC_FP64, 8>()
               : W == 4 ? persistent_fn<MC_PREC_FP64, 4>()
               : W == 2 ? persistent_fn<MC_PREC_FP64, 2>()
                        : persistent_fn<MC_PREC_FP64, 1>();
    return W == 8 ? persistent_fn<MC_PREC_FP32, 8>()
           : W == 4 ? persistent_fn<MC_PREC_FP32, 4>()
           : W == 2 ? persistent_fn<MC_PREC_FP32, 2>()
                    : persistent_fn<MC_PREC_FP32, 1>();
}

int persistent_grid(const DevState &d, int warps_per_cell, int max_blocks)
{
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return 0;
    const size_t sm = phase_smem_bytes(d.stencil_cap, warps_per_cell);
    const int nt = warps_per_cell > 4 ? 32 * warps_per_cell : BLOCK;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel(d.precision, warps_per_cell), nt, sm) !=
        cudaSuccess)
        return 0;
    // one block per group of active cells: blocks without a cell would only
    // add arrivals to every grid barrier
    const int cpb = nt / (32 * warps_per_cell);
    const int needed = std::max((d.n_act + cpb - 1) / cpb, 32);
    return std::max(0, std::min(std::min(per_sm * sms, needed), max_blocks));
}

int launch_persistent(const DevState &d, int buf, int n_sweeps, int warps_per_cell, int grid, unsigned int *bar,
                      int *scan_tot, cudaStream_t st)
{
    const size_t sm = phase_smem_bytes(d.stencil_cap, warps_per_cell);
    GridBar gb{bar, scan_tot};
    DevState dd = d;
    void *args[] = {(void *)&dd, (void *)&buf, (void *)&n_sweeps, (void *)&gb};
    const int nt = warps_per_cell > 4 ? 32 * warps_per_cell : BLOCK;
    const cudaError_t e = cudaLaunchCooperativeKernel(persistent_kernel(d.precision, warps_per_cell), dim3(grid),
                                                      dim3(nt), args, sm, st);
    return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace flipmc
