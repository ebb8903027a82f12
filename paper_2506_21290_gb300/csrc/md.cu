// Molecular dynamics of the flexible three-site molecules (Sec. II.D: NVT,
// time step 0.001, Nose-Hoover thermostat with relaxation time 1), FP64.
//
// One step, a symmetric (time-reversible) splitting of velocity Verlet and
// the thermostat, m = 1, g = 3N degrees of freedom, Q = g T tau^2:
//   xi += dt/2 (2K - gT) / Q;  eta += dt/2 xi;  v *= exp(-xi dt/2);  v += dt/2 F
//   q  += rint(v dt / h)                     (fixed point, periodic images counted)
//   cell list; F = forces (Eq. 1 and 2, every pair inside its range)
//   v += dt/2 F;  v *= exp(-xi dt/2);  xi += dt/2 (2K - gT) / Q;  eta += dt/2 xi
// K is the kinetic energy sum v^2 / 2 over the replica, in a fixed order
// (chunks of kMdChunk atoms, then the chunk sums).  The
// conserved quantity is K + U + Q xi^2 / 2 + g T eta.
#include "flipmc_device.cuh"
#include "md.h"

namespace flipmc {

namespace {

constexpr int MD_BLOCK = 256;

}  // namespace

// Partial kinetic energy of one chunk of kMdChunk atoms (one replica's): each
// thread its atoms in order, then a fixed tree.
__global__ void __launch_bounds__(MD_BLOCK) md_kin_partial_kernel(MdDev m)
{
    const int a0 = m.chunk_a0[blockIdx.x], a1 = m.chunk_a0[blockIdx.x + 1];
    double s = 0.0;
    for (int i = a0 + threadIdx.x; i < a1; i += MD_BLOCK) {
        const double *v = m.v + 3 * (size_t)i;
        s = __dadd_rn(s, __dadd_rn(__dadd_rn(__dmul_rn(v[0], v[0]), __dmul_rn(v[1], v[1])), __dmul_rn(v[2], v[2])));
    }
    __shared__ double red[MD_BLOCK];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = MD_BLOCK / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) m.part[blockIdx.x] = red[0];
}

// Per replica (one block): K from the chunk sums (strided, fixed tree), then
// xi += dt/2 (2K - gT)/Q, eta += dt/2 xi, and the scale exp(-xi dt/2).
__global__ void __launch_bounds__(128) md_thermo_kernel(DevState d, MdDev m)
{
    const int r = blockIdx.x;
    double s = 0.0;
    for (int k = m.rep_chunk0[r] + threadIdx.x; k < m.rep_chunk0[r + 1]; k += 128) s = __dadd_rn(s, m.part[k]);
    __shared__ double red[128];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double K = 0.5 * red[0];
    const double g = 3.0 * (double)d.rep[r].n_sites;
    const double xi = __dadd_rn(m.xi[r], __dmul_rn(m.hdt, __ddiv_rn(__dsub_rn(2.0 * K, g * m.T[r]), m.Q[r])));
    m.xi[r] = xi;
    m.eta[r] = __dadd_rn(m.eta[r], __dmul_rn(m.hdt, xi));
    m.K[r] = K;
    m.scale[r] = exp(-xi * m.hdt);
}

// Velocity components: BEGIN: v = v s + dt/2 F; END: v = (v + dt/2 F) s.
template <bool BEGIN>
__global__ void md_kick_kernel(DevState d, MdDev m)
{
    const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 3 * (size_t)d.n_sites) return;
    const double sc = m.scale[d.rep_of_site[j / 3]];
    m.v[j] = BEGIN ? __dadd_rn(__dmul_rn(m.v[j], sc), __dmul_rn(m.hdt, m.F[j]))
                   : __dmul_rn(__dadd_rn(m.v[j], __dmul_rn(m.hdt, m.F[j])), sc);
}

__global__ void md_drift_kernel(DevState d, int buf, MdDev m)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= d.n_sites) return;
    const int r = d.rep_of_site[g];
    const RepInfo ri = d.rep[r];
    int4 rc = d.rec[buf][g];
    const int site = ri.site_off + rec_site(rc.w);
    const double s = m.dt * ri.inv_h;   // fixed-point units per unit velocity and step
    uint32_t q3[3] = {(uint32_t)rc.x, (uint32_t)rc.y, (uint32_t)rc.z};
    for (int ax = 0; ax < 3; ++ax) {
        const long long step = (long long)rint(__dmul_rn(m.v[3 * (size_t)site + ax], s));
        const long long moved = (long long)q3[ax] + step;
        if (moved < 0) d.img[3 * site + ax] -= 1;
        else if (moved >= 4294967296ll) d.img[3 * site + ax] += 1;
        q3[ax] = (uint32_t)moved;
    }
    rc.x = (int)q3[0];
    rc.y = (int)q3[1];
    rc.z = (int)q3[2];
    d.rec[buf][g] = rc;
}

// The pair factor (-r dphi/dr) / r^2 in FP32: r^2 from the exact int32
// differences (one rounding per axis), the derivative of Eq. 1 and Eq. 2.
__device__ __forceinline__ float virial_over_r2_f32(const ModelDev &md, float r2, int ab, bool bonded)
{
    const float inv = 1.0f / r2;
    float w = 0.f;
    if (r2 < md.rc2f[ab]) {
        const float t = md.s2f[ab] * inv;
        const float s6 = t * t * t;
        w = 6.0f * md.e4f * s6 * (2.0f * s6 - 1.0f);
    }
    if (bonded) {
        const float x = r2 * md.invR2f[ab];
        w += 2.0f * md.nkef * x / (1.0f - x);
    }
    return w * inv;
}

// F_i = sum over partners j of (-r dphi/dr) / r^2 (x_i - x_j), partners in
// the neighbour cells in cell order, then record order; FP64, or FP32 terms
// summed in FP32 (FP32 = true).
template <bool FP32>
__global__ void md_force_kernel(DevState d, int buf, MdDev m)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= d.n_sites) return;
    const int r = d.rep_of_site[g];
    const RepInfo ri = d.rep[r];
    const ModelDev &md = *d.model;
    const int4 me = d.rec[buf][g];
    const int si = rec_site(me.w), ti = rec_type(me.w), mi = rec_mol(me.w);
    const int nc = ri.nc;
    const uint32_t *shift = d.ctr[r].shift;
    const int cx = (int)cell_axis((uint32_t)me.x, shift[0], nc);
    const int cy = (int)cell_axis((uint32_t)me.y, shift[1], nc);
    const int cz = (int)cell_axis((uint32_t)me.z, shift[2], nc);
    float rc2max = 0.f;
    for (int k = 0; k < 9; ++k) rc2max = fmaxf(rc2max, md.rc2f[k]);
    const float pre = rc2max * 1.01f;
    const bool small = nc == 2;
    const int ns = small ? 8 : 27;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    for (int k = 0; k < ns; ++k) {
        int ox, oy, oz;
        if (small) {
            ox = k & 1; oy = (k >> 1) & 1; oz = k >> 2;
        } else {
            ox = k % 3 - 1; oy = (k / 3) % 3 - 1; oz = k / 9 - 1;
        }
        const int c = ri.cell_off + (((cz + oz + nc) % nc) * nc + (cy + oy + nc) % nc) * nc + (cx + ox + nc) % nc;
        const int s0 = d.cell_start[c], s1 = d.cell_start[c + 1];
        for (int j = s0; j < s1; ++j) {
            const int4 o = d.rec[buf][j];
            if (rec_site(o.w) == si) continue;
            const int dx = (int)((uint32_t)o.x - (uint32_t)me.x);
            const int dy = (int)((uint32_t)o.y - (uint32_t)me.y);
            const int dz = (int)((uint32_t)o.z - (uint32_t)me.z);
            const bool bonded = rec_mol(o.w) == mi;
            if (!bonded) {
                const float ex = (float)dx * ri.hf, ey = (float)dy * ri.hf, ez = (float)dz * ri.hf;
                if (ex * ex + ey * ey + ez * ez > pre) continue;
            }
            if (FP32) {
                const float ex = (float)dx * ri.hf, ey = (float)dy * ri.hf, ez = (float)dz * ri.hf;
                const float w = virial_over_r2_f32(md, fmaf(ex, ex, fmaf(ey, ey, ez * ez)), 3 * ti + rec_type(o.w),
                                                   bonded);
                gx = fmaf(-w, ex, gx);
                gy = fmaf(-w, ey, gy);
                gz = fmaf(-w, ez, gz);
            } else {
                const double r2 = r2_fixed64(dx, dy, dz, ri.h);
                const double w = virial_over_r2(md, r2, 3 * ti + rec_type(o.w), bonded);
                fx = __dsub_rn(fx, __dmul_rn(w, __dmul_rn((double)dx, ri.h)));
                fy = __dsub_rn(fy, __dmul_rn(w, __dmul_rn((double)dy, ri.h)));
                fz = __dsub_rn(fz, __dmul_rn(w, __dmul_rn((double)dz, ri.h)));
            }
        }
    }
    double *F = m.F + 3 * (size_t)(ri.site_off + si);
    F[0] = FP32 ? (double)gx : fx;
    F[1] = FP32 ? (double)gy : fy;
    F[2] = FP32 ? (double)gz : fz;
}

void launch_md_begin(const DevState &d, const MdDev &m, cudaStream_t st)
{
    md_kin_partial_kernel<<<m.n_chunks, MD_BLOCK, 0, st>>>(m);
    md_thermo_kernel<<<d.n_rep, 128, 0, st>>>(d, m);
    md_kick_kernel<true><<<(unsigned)((3 * (size_t)d.n_sites + 255) / 256), 256, 0, st>>>(d, m);
}

void launch_md_drift(const DevState &d, int buf, const MdDev &m, cudaStream_t st)
{
    md_drift_kernel<<<(d.n_sites + 255) / 256, 256, 0, st>>>(d, buf, m);
}

void launch_md_forces(const DevState &d, int buf, const MdDev &m, cudaStream_t st)
{
    if (m.fp32_forces) md_force_kernel<true><<<(d.n_sites + 255) / 256, 256, 0, st>>>(d, buf, m);
    else md_force_kernel<false><<<(d.n_sites + 255) / 256, 256, 0, st>>>(d, buf, m);
}

void launch_md_end(const DevState &d, const MdDev &m, cudaStream_t st)
{
    md_kick_kernel<false><<<(unsigned)((3 * (size_t)d.n_sites + 255) / 256), 256, 0, st>>>(d, m);
    md_kin_partial_kernel<<<m.n_chunks, MD_BLOCK, 0, st>>>(m);
    md_thermo_kernel<<<d.n_rep, 128, 0, st>>>(d, m);
}


}  // namespace flipmc
