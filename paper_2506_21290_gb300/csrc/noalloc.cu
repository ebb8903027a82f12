// mc_energy_noalloc: the FP64 total energy of one configuration that already
// sits in the caller's device memory, computed without allocating any device
// memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool (which owns the device memory and must not be
// bypassed), code under a fixed device-memory budget, or embedded callers that
// are only allowed to enqueue kernels on a stream they were handed.  For them
// the working space of the cell-list build and of the energy reduction lives
// in one file-scope __device__ array, sized for up to kMaxSites atoms and
// kMaxCells cells.  Every GPU that loads this library holds that array (about
// 3.5 MB) until the process exits.  The first call on a device looks up the
// array's device address (cudaGetSymbolAddress, with that device current);
// make that first call before any stream capture.
//
// The array is shared by all calls on a device and keeps the last call's
// contents; everything a call relies on starting at zero is cleared by that
// call.  Two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array and give undefined results:
// serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/flipmc.h"
#include "cell_list.h"
#include "energy.h"
#include "flipmc_types.h"

using namespace flipmc;

namespace {

constexpr int kMaxSites = 1 << 16;   // atoms per call
constexpr int kMaxCells = 1 << 15;   // cells per call
constexpr int kMaxDevices = 64;

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// byte offsets inside the scratch array
constexpr size_t kOffRep = 0;
constexpr size_t kOffPar = al256(kOffRep + sizeof(RepInfo));
constexpr size_t kOffCtr = al256(kOffPar + sizeof(RepParam));
constexpr size_t kOffModel = al256(kOffCtr + sizeof(RepCtr));
constexpr size_t kOffMix = al256(kOffModel + sizeof(ModelDev));
constexpr size_t kOffActOff = al256(kOffMix + sizeof(MixDev));
constexpr size_t kOffErr = al256(kOffActOff + 2 * sizeof(int));
constexpr size_t kOffRepOfSite = al256(kOffErr + sizeof(int));
constexpr size_t kOffRec0 = al256(kOffRepOfSite + sizeof(int) * kMaxSites);
constexpr size_t kOffRec1 = al256(kOffRec0 + sizeof(int4) * kMaxSites);
constexpr size_t kOffCount = al256(kOffRec1 + sizeof(int4) * kMaxSites);
constexpr size_t kOffStart = al256(kOffCount + sizeof(int) * kMaxCells);
constexpr size_t kOffCellOf = al256(kOffStart + sizeof(int) * (kMaxCells + 1));
constexpr size_t kOffSlotOf = al256(kOffCellOf + sizeof(int) * kMaxSites);
constexpr size_t kOffESite = al256(kOffSlotOf + sizeof(int) * kMaxSites);
constexpr size_t kScratchBytes = al256(kOffESite + sizeof(double) * kMaxSites);
static_assert(kMaxCells <= kMaxSites, "the partial-sum region holds one double per cell");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// errors go where mc_last_error() reads them
int noalloc_fail(int code, const char *msg)
{
    return record_error(code, msg);
}

// Per device, the device address of the scratch array, looked up once with
// that device current (the host-side name of the array is only a stand-in).
std::mutex g_addr_mu;
unsigned char *g_addr[kMaxDevices] = {};

int scratch_address(int dev, unsigned char **out)
{
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
            return noalloc_fail(MC_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
        g_addr[dev] = (unsigned char *)p;
    }
    *out = g_addr[dev];
    return MC_OK;
}

// The call's constants, passed by value as a kernel parameter: the call then
// copies nothing from host memory (a copy from pageable host memory can wait
// for the stream before it returns).
struct Header {
    RepInfo rep;
    RepParam par;
    RepCtr ctr;
    ModelDev model;
    int act_off[2];
};

// one block: the constants into the scratch array, the error word and the
// per-site replica index cleared
__global__ void noalloc_init_kernel(Header hd, unsigned char *base, int n_sites)
{
    if (threadIdx.x == 0) {
        *(RepInfo *)(base + kOffRep) = hd.rep;
        *(RepParam *)(base + kOffPar) = hd.par;
        *(RepCtr *)(base + kOffCtr) = hd.ctr;
        *(ModelDev *)(base + kOffModel) = hd.model;
        ((int *)(base + kOffActOff))[0] = hd.act_off[0];
        ((int *)(base + kOffActOff))[1] = hd.act_off[1];
        *(int *)(base + kOffErr) = 0;
    }
    int *rep_of_site = (int *)(base + kOffRepOfSite);
    for (int i = threadIdx.x; i < n_sites; i += blockDim.x) rep_of_site[i] = 0;
}

// records {q, w} in site order from the caller's arrays; a type outside
// {0,1,2} sets the error word
__global__ void noalloc_pack_kernel(const uint32_t *q, const int32_t *types, int n, int4 *rec, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = types[i];
    if (t < 0 || t > 2) atomicOr(err, 1);
    rec[i] = make_int4((int)q[3 * i], (int)q[3 * i + 1], (int)q[3 * i + 2], ((i / 3) << 4) | ((i % 3) << 2) | (t & 3));
}

// an invalid input gives NaN rather than a number that looks valid
__global__ void noalloc_poison_kernel(const int *err, double *out)
{
    if (threadIdx.x == 0 && *err) out[0] = __longlong_as_double(0x7FF8000000000000ll);
}

}  // namespace

extern "C" int mc_energy_noalloc(double L, int n_mol, const uint32_t *dev_q, const int32_t *dev_types,
                                 const mc_params *params, double *dev_E_out, void *stream)
{
    if (n_mol < 1 || !dev_q || !dev_types || !dev_E_out) return noalloc_fail(MC_ERR_INVALID_ARG, "bad argument");
    if (!(L > 0.0) || !std::isfinite(L)) return noalloc_fail(MC_ERR_INVALID_ARG, "box side must be positive");
    if ((long long)n_mol * 3 > kMaxSites)
        return noalloc_fail(MC_ERR_INVALID_ARG, "mc_energy_noalloc holds at most 65536 atoms (21845 molecules)");
    mc_params p;
    if (params) {
        p = *params;
    } else {
        p.sigma[0] = 0.9;
        p.sigma[1] = 1.0;
        p.sigma[2] = 1.1;
        p.eps = 1.0;
        p.fene_k = 33.75;
        p.fene_r0 = 1.5;
    }
    for (int k = 0; k < 3; ++k)
        if (!(p.sigma[k] > 0.0)) return noalloc_fail(MC_ERR_INVALID_ARG, "sigma must be positive");
    // the types are on the device: cells must cover a bond between any two types
    double smax = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) smax = std::fmax(smax, 0.5 * (p.sigma[a] + p.sigma[b]));
    const double range = std::fmax(std::pow(2.0, 1.0 / 6.0) * smax, p.fene_r0 * smax);
    if (L < 2.0 * range) return noalloc_fail(MC_ERR_INVALID_ARG, "box side smaller than twice the interaction range");
    const double two32 = 4294967296.0;
    int nc = 2;
    while (std::floor(two32 / (nc + 2)) * (L / two32) >= range && nc + 2 <= 1024) nc += 2;
    while ((long long)nc * nc * nc > kMaxCells) nc -= 2;
    const int n_sites = 3 * n_mol;
    const int n_cells = nc * nc * nc;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(MC_ERR_NO_DEVICE, "no current CUDA device");
    unsigned char *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    Header hd;
    std::memset(&hd, 0, sizeof hd);
    hd.rep.n_sites = n_sites;
    hd.rep.nc = nc;
    hd.rep.L = L;
    hd.rep.h = L / two32;
    hd.rep.inv_h = two32 / L;
    hd.rep.hf = (float)hd.rep.h;
    hd.par.T = 1.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const int ab = 3 * a + b;
            const double s = (p.sigma[a] + p.sigma[b]) * 0.5;
            const double R = p.fene_r0 * s;
            hd.model.s2[ab] = s * s;
            hd.model.rc2[ab] = 0x1.428a2f98d728bp+0 * (s * s);
            hd.model.R2[ab] = R * R;
            hd.model.s2f[ab] = (float)hd.model.s2[ab];
            hd.model.rc2f[ab] = (float)hd.model.rc2[ab];
            hd.model.R2f[ab] = (float)hd.model.R2[ab];
            hd.model.invR2f[ab] = (float)(1.0 / hd.model.R2[ab]);
        }
    hd.model.eps = p.eps;
    hd.model.e4 = 4.0 * p.eps;
    hd.model.ke = p.fene_k * p.eps;
    hd.model.nke = -hd.model.ke;
    hd.act_off[0] = 0;
    hd.act_off[1] = (nc / 2) * (nc / 2) * (nc / 2);

    DevState d{};
    d.n_rep = 1;
    d.n_sites = n_sites;
    d.n_cells = n_cells;
    d.n_act = hd.act_off[1];
    d.precision = MC_PREC_FP64;
    d.rep = (const RepInfo *)(base + kOffRep);
    d.par = (const RepParam *)(base + kOffPar);
    d.ctr = (RepCtr *)(base + kOffCtr);
    d.model = (const ModelDev *)(base + kOffModel);
    d.mix = (const MixDev *)(base + kOffMix);
    d.act_off = (const int *)(base + kOffActOff);
    d.err = (int *)(base + kOffErr);
    d.rep_of_site = (const int *)(base + kOffRepOfSite);
    d.rec[0] = (int4 *)(base + kOffRec0);
    d.rec[1] = (int4 *)(base + kOffRec1);
    d.cell_count = (int *)(base + kOffCount);
    d.cell_start = (int *)(base + kOffStart);
    d.cell_of = (int *)(base + kOffCellOf);
    d.slot_of = (int *)(base + kOffSlotOf);
    double *e_part = (double *)(base + kOffESite);   // per-cell partial sums

    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    };
    noalloc_init_kernel<<<1, 256, 0, st>>>(hd, base, n_sites);
    chk(cudaGetLastError());
    noalloc_pack_kernel<<<(n_sites + 255) / 256, 256, 0, st>>>(dev_q, dev_types, n_sites, d.rec[0], d.err);
    chk(cudaGetLastError());
    launch_cell_list(d, 0, 1, st);
    chk(cudaGetLastError());
    launch_energy(d, 1, e_part, dev_E_out, st);
    chk(cudaGetLastError());
    noalloc_poison_kernel<<<1, 32, 0, st>>>(d.err, dev_E_out);
    chk(cudaGetLastError());
    if (e != cudaSuccess) return noalloc_fail(MC_ERR_CUDA, (std::string("mc_energy_noalloc: ") + cudaGetErrorString(e)).c_str());
    return MC_OK;
}
