// Device-side building blocks of the flip Monte Carlo library (sm_103a).
//
// Model of arXiv 2506.21290 Sec. II.A: WCA on every pair (Eq. 1), FENE on the
// three bonds of each molecule (Eq. 2), Philox4x32-10 counter-based random
// numbers (Salmon et al., SC'11).
//
// The FP64 functions here use explicit round-to-nearest intrinsics
// (__dadd_rn, __dmul_rn, __ddiv_rn, ...) so that no multiply-add is fused:
// each operation rounds once, in the order written, which is what makes the
// FP64 mode reproduce a host FP64 evaluation of the same expressions exactly.
#pragma once

#include <cstdint>

#include "flipmc_types.h"

namespace flipmc {

// ---------------------------------------------------------------------------
// Philox4x32-10: ten rounds, each two 32x32->64 multiplies by the Philox
// constants, the high halves xor-ed with the other counter words and the key;
// the key is advanced by the Weyl increments before every round but the first.
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t a = (uint64_t)0xD2511F53u * c.x;
        const uint64_t b = (uint64_t)0xCD9E8D57u * c.z;
        U4 n;
        n.x = (uint32_t)(b >> 32) ^ c.y ^ k0;
        n.y = (uint32_t)b;
        n.z = (uint32_t)(a >> 32) ^ c.w ^ k1;
        n.w = (uint32_t)a;
        c = n;
    }
    return c;
}

// Random block number `word0` of cell `cell` in sweep `sweep` under `seed`.
__host__ __device__ __forceinline__ U4 rng_block(uint32_t word0, uint32_t cell, uint64_t sweep, uint64_t seed)
{
    U4 c{word0, cell, (uint32_t)sweep, (uint32_t)(sweep >> 32)};
    return philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// ---------------------------------------------------------------------------
// FP64 natural logarithm, atanh series: x = m 2^e with m folded into
// [sqrt(1/2), sqrt(2)], z = (m-1)/(m+1), ln x = e ln2 + 2 sum_k z^(2k+1)/(2k+1),
// twelve terms (|z| <= 0.1716).  Each operation rounds to nearest, unfused.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ln_series(double x)
{
    if (!(x > 0.0)) return (x == 0.0) ? -__longlong_as_double(0x7FF0000000000000ll) : __longlong_as_double(0x7FF8000000000000ll);
    if (x == __longlong_as_double(0x7FF0000000000000ll)) return x;
    unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0) {
        x = __dmul_rn(x, 18446744073709551616.0);   // 2^64
        bits = (unsigned long long)__double_as_longlong(x);
        e = (int)((bits >> 52) & 0x7FF) - 64;
    }
    e -= 1023;
    double m = __longlong_as_double((long long)((bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
    if (m > 0x1.6a09e667f3bcdp+0) {      // fold (sqrt2, 2) onto (sqrt(1/2), 1)
        m = __dmul_rn(m, 0.5);
        e = e + 1;
    }
    const double z = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double w = __dmul_rn(z, z);
    double s = 2.0 / 23.0;
    s = __dadd_rn(__dmul_rn(s, w), 2.0 / 21.0);
    s = __dadd_rn(__dmul_rn(s, w), 2.0 / 19.0);
    s = __dadd_rn(__dmul_rn(s, w), 2.0 / 17.0);
    s = __dadd_rn(__dmul_rn(s, w), 2.0 / 15.0);
    s = __dadd_rn(__dmul_rn(s, w), 2.0 / 13.0);
    s = __dadd_rn(__dmul_rn(s, w), 2.0 / 11.0);
    s = __dadd_rn(__dmul_rn(s, w), 2.0 / 9.0);
    s = __dadd_rn(__dmul_rn(s, w), 2.0 / 7.0);
    s = __dadd_rn(__dmul_rn(s, w), 2.0 / 5.0);
    s = __dadd_rn(__dmul_rn(s, w), 2.0 / 3.0);
    s = __dadd_rn(__dmul_rn(s, w), 2.0);
    const double series = __dmul_rn(z, s);
    const double el = __dmul_rn((double)e, 0x1.62e42fefa39efp-1);   // double nearest ln 2
    return __dadd_rn(el, series);
}

// ---------------------------------------------------------------------------
// Pair potentials.  Type pair index ab = 3a + b.
// ---------------------------------------------------------------------------

// r2 of a fixed-point pair: int32 differences (the minimum image) times h.
__device__ __forceinline__ double r2_fixed64(int dx, int dy, int dz, double h)
{
    const double x = __dmul_rn((double)dx, h);
    const double y = __dmul_rn((double)dy, h);
    const double z = __dmul_rn((double)dz, h);
    return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
}

// WCA (Eq. 1) in FP64: 4 eps ((s2/r2)^6 - (s2/r2)^3) + eps inside the cutoff.
__device__ __forceinline__ double wca64(const ModelDev &md, double r2, int ab)
{
    if (!(r2 < md.rc2[ab])) return 0.0;
    const double t = __ddiv_rn(md.s2[ab], r2);
    const double s6 = __dmul_rn(__dmul_rn(t, t), t);
    return __dadd_rn(__dmul_rn(md.e4, __dsub_rn(__dmul_rn(s6, s6), s6)), md.eps);
}

// FENE (Eq. 2) in FP64: -K eps ln(1 - r2/R2).
__device__ __forceinline__ double fene64(const ModelDev &md, double r2, int ab)
{
    const double x = __ddiv_rn(r2, md.R2[ab]);
    return __dmul_rn(md.nke, ln_series(__dsub_rn(1.0, x)));
}

__device__ __forceinline__ double phi64(const ModelDev &md, double r2, int ab, bool bonded)
{
    double u = wca64(md, r2, ab);
    if (bonded) u = __dadd_rn(u, fene64(md, r2, ab));
    return u;
}

// Pair virial -r dphi/dr in FP64 (the derivative of Eq. 1 and Eq. 2):
// WCA 24 eps s6 (2 s6 - 1) inside the cutoff (s6 = (sigma^2/r^2)^3), and for a
// bond FENE -2 K eps x / (1 - x) with x = r^2 / (R0 sigma)^2.
__device__ __forceinline__ double virial64(const ModelDev &md, double r2, int ab, bool bonded)
{
    double w = 0.0;
    if (r2 < md.rc2[ab]) {
        const double t = __ddiv_rn(md.s2[ab], r2);
        const double s6 = __dmul_rn(__dmul_rn(t, t), t);
        w = __dmul_rn(__dmul_rn(6.0, md.e4), __dmul_rn(s6, __dsub_rn(__dmul_rn(2.0, s6), 1.0)));
    }
    if (bonded) {
        const double x = __ddiv_rn(r2, md.R2[ab]);
        w = __dadd_rn(w, __dmul_rn(__dmul_rn(2.0, md.nke), __ddiv_rn(x, __dsub_rn(1.0, x))));
    }
    return w;
}

// The same pair virial divided by r^2 (the force factor: F_i += w (x_i - x_j)),
// with one FP64 division for the WCA term.
__device__ __forceinline__ double virial_over_r2(const ModelDev &md, double r2, int ab, bool bonded)
{
    const double inv = __ddiv_rn(1.0, r2);
    double w = 0.0;
    if (r2 < md.rc2[ab]) {
        const double t = __dmul_rn(md.s2[ab], inv);
        const double s6 = __dmul_rn(__dmul_rn(t, t), t);
        w = __dmul_rn(__dmul_rn(6.0, md.e4), __dmul_rn(s6, __dsub_rn(__dmul_rn(2.0, s6), 1.0)));
    }
    if (bonded) {
        const double x = __ddiv_rn(r2, md.R2[ab]);
        w = __dadd_rn(w, __dmul_rn(__dmul_rn(2.0, md.nke), __ddiv_rn(x, __dsub_rn(1.0, x))));
    }
    return __dmul_rn(w, inv);
}

// FP32 WCA with its magnitude 4eps s12 + 4eps s6 + eps (the FP32 error scale).
__device__ __forceinline__ void wca32(const ModelDev &md, float r2, int ab, float &u, float &mag)
{
    const float t = __fdividef(md.s2f[ab], r2);
    const float s6 = t * t * t;
    const float a = md.e4f * s6;
    u = fmaf(a, s6, md.epsf - a);
    mag = fmaf(a, s6, a + md.epsf);
}

// FP32 FENE with its magnitude K eps (|ln(1-x)| + x/(1-x) + 1).
__device__ __forceinline__ void fene32(const ModelDev &md, float r2, int ab, float &u, float &mag)
{
    const float x = r2 * md.invR2f[ab];
    const float y = 1.0f - x;
    const float l = __logf(y);
    u = md.nkef * l;
    mag = md.kef * (fabsf(l) + __fdividef(x, y) + 1.0f);
}

// ---------------------------------------------------------------------------
// Fixed-point helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cell_axis(uint32_t q, uint32_t shift, int nc)
{
    return (uint32_t)(((uint64_t)(uint32_t)(q + shift) * (uint64_t)nc) >> 32);
}

__device__ __forceinline__ int cell_local(uint32_t qx, uint32_t qy, uint32_t qz, const uint32_t *shift, int nc)
{
    const int cx = (int)cell_axis(qx, shift[0], nc);
    const int cy = (int)cell_axis(qy, shift[1], nc);
    const int cz = (int)cell_axis(qz, shift[2], nc);
    return (cz * nc + cy) * nc + cx;
}

__device__ __forceinline__ int32_t uniform_disp(uint32_t w, int32_t D)
{
    const uint64_t span = (uint64_t)(2 * (int64_t)D + 1);
    return (int32_t)((int64_t)(((uint64_t)w * span) >> 32) - D);
}

__device__ __forceinline__ int move_type(uint32_t w, const MixDev &mx)
{
    if ((uint64_t)w < mx.thr[0]) return MC_MOVE_ATOM;
    if ((uint64_t)w < mx.thr[1]) return MC_MOVE_FLIP;
    if ((uint64_t)w < mx.thr[2]) return MC_MOVE_MOL_TRANS;
    return MC_MOVE_MOL_ROT;
}

// record word w = (molecule << 4) | (slot << 2) | type
__device__ __forceinline__ int rec_mol(int w) { return (int)((uint32_t)w >> 4); }
__device__ __forceinline__ int rec_slot(int w) { return (w >> 2) & 3; }
__device__ __forceinline__ int rec_type(int w) { return w & 3; }
__device__ __forceinline__ int rec_site(int w) { return 3 * rec_mol(w) + rec_slot(w); }

// binary search: largest r with off[r] <= x (off has n+1 entries, off[0] = 0)
__device__ __forceinline__ int find_segment(const int *off, int n, int x)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

}  // namespace flipmc
