// Structures shared by the host engine and the device kernels.
#pragma once

#include <cstdint>

#include "../../include/flipmc.h"

namespace flipmc {

// Potential tables, type pair ab = 3a + b (Eq. 1-2).
struct ModelDev {
    double s2[9];    // sigma_ab^2
    double rc2[9];   // (2^(1/3)) sigma_ab^2: WCA cutoff squared
    double R2[9];    // (R0 sigma_ab)^2: FENE divergence squared
    double eps, e4, nke, ke;
    float s2f[9], rc2f[9], R2f[9], invR2f[9];
    float epsf, e4f, nkef, kef;
    float bond_guard_f;   // FP32 bond-length ratio beyond which FP32 defers to FP64
    float recheck_gap_f;
};

// Move-mix parameters of the current sweep call.
struct MixDev {
    uint64_t thr[3];      // move-type thresholds on a 32-bit word
    double rot_a;
};

// Per-replica static layout.
struct RepInfo {
    int n_sites;
    int site_off;    // first global site
    int nc;          // cells per axis
    int cell_off;    // first global cell
    int act_off;     // first global active-cell slot within a colour
    int pad;
    double L, h, inv_h;
    float hf;
    float h2f;       // h^2 rounded to FP32
    float pre_r2;    // screening radius squared (sigma units): 1.01 x the largest WCA cutoff squared, FP32
    float r2q;       // the same in fixed-point units squared: pre_r2 / h2f
    float rconf;     // conflict radius squared, fixed-point units: rc2max x 1.0201 / h2f
};

// Per-replica parameters of the current sweep call (written by the host).
struct RepParam {
    double T;
    uint64_t seed;
    int32_t D_atom;      // atom step half-width in fixed-point units
    int32_t D_mol;       // molecule step half-width in fixed-point units
    float T32;           // T rounded to FP32
    int32_t pad;
};

// Per-replica counters owned by the device.
struct RepCtr {
    uint64_t sweep;      // number of the sweep being (or next to be) run
    uint32_t shift[4];   // grid shift of that sweep (x, y, z)
};

// Staging of a cell neighbourhood: padding candidates after the staged atoms
// (far away, record word kPadWord: type 0 and a molecule index no atom has,
// since replicas hold fewer than 2^27 - 1 molecules).
constexpr int kPadSlots = 4;
constexpr int kPadWord = 0x7FFFFFF0;
constexpr int kMaxMolecules = (1 << 27) - 2;

// counters per replica (uint64)
enum {
    STAT_ATT = 0,       // [4]
    STAT_ACC = 4,       // [4]
    STAT_REJ_GEOM = 8,
    STAT_REJ_BOND = 9,
    STAT_PAIRS = 10,
    STAT_RECHECK = 11,
    STAT_SWEEPS = 12,
    STAT_INTER = 13,    // pair-potential evaluations inside their range (WCA r < r_c, FENE), old and new
    STAT_RECOMP = 14,   // FP64 recomputes of the total energy (recompute_every)
    STAT_N = 16
};

// error bits
enum {
    ERR_STENCIL = 1,    // neighbourhood larger than the staging capacity
    ERR_TERMS = 2,      // FP64 ordered-sum buffer overflow
    ERR_TIMEOUT = 4,
};

// Everything a kernel needs, by value.
struct DevState {
    int n_rep;
    int n_sites;         // total over replicas
    int n_cells;         // total over replicas
    int n_act;           // active cells per colour, total over replicas
    int stencil_cap;     // atoms staged per neighbourhood (plus kPadSlots padding candidates)
    int precision;
    unsigned wait_limit; // polls after which a wait between blocks gives up (0: the defaults)
    const RepInfo *rep;
    const RepParam *par;
    RepCtr *ctr;
    const ModelDev *model;
    const MixDev *mix;
    const int *rep_of_site;
    const int *act_off;  // n_rep + 1 prefix of (nc/2)^3
    const int2 *act_slot;    // per active-cell slot of a colour (n_act), in schedule order: {replica, active
                             // cell within the replica}; null for one replica (slot = active cell)
    int4 *rec[2];        // double-buffered records {qx, qy, qz, w}, cell-sorted
    int *cell_count;
    int *cell_count2;    // second count buffer (persistent launch: sweep s + 1 is counted while sweep s finishes)
    int *cell_start;     // n_cells + 1
    int *scan_part;      // ceil(n_cells / 1024) + 1 block totals of the multi-block scan (nullable: one block)
    int *cell_of;
    int *slot_of;
    int *img;            // 3 per site, indexed by global site index
    double *cell_dE;     // accepted Delta E per cell in the last sweep
    uint4 *att_rnd;      // 2 per record slot: the 8 random words of the slot's attempt (nullable)
    float *att_thr32;    // per record slot: FP32 threshold -T ln u (FP32 mode)
    double *att_thr64;   // per record slot: FP64 threshold (FP64 mode)
    unsigned long long *stats;   // STAT_N per replica
    double *e_run;       // per replica
    int *err;
    unsigned int *cell_done;     // per cell: colour phases it completed in the current persistent launch
};

}  // namespace flipmc
