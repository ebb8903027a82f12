// Host engine behind the C ABI of include/flipmc.h.
//
// A handle owns all device memory of one batch of replicas (a single replica
// is a batch of one).  State lives on the device as cell-sorted 16-byte
// records {qx, qy, qz, w}, w = (molecule << 4) | (slot << 2) | type, in two
// buffers: each sweep's cell-list build reads one and writes the other.  One
// sweep (cell list + 8 colour phases + finalisation) is captured once per
// buffer parity as a CUDA graph and replayed; everything a sweep reads that can
// change between calls (T, seed, move mix, sweep counter) sits in device
// memory, so the graphs never need re-capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/flipmc.h"
#include "cell_list.h"
#include "energy.h"
#include "flipmc_types.h"
#include "md.h"

using namespace flipmc;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define CUDA_TRY(expr)                                                                              \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess)                                                                      \
            return fail(MC_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));           \
    } while (0)

const double kCbrt2 = 0x1.428a2f98d728bp+0;   // double nearest 2^(1/3)
const double kTwo32 = 4294967296.0;
const int kMaxPersistentBlocks = 8192;

// x -> floor(frac(x / L) * 2^32), the library's quantisation of positions
uint32_t quantize(double x, double L)
{
    double t = x / L;
    t = t - std::floor(t);
    double v = std::floor(t * kTwo32);
    if (v >= kTwo32) v = 0.0;
    return (uint32_t)v;
}

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

// mc_test_fail_alloc: allocations left before the one that fails (-1: off)
std::atomic<int> g_fail_alloc{-1};

// f(begin, end) over [0, n) in contiguous chunks of at least `grain` items, on
// up to 16 host threads (the calling thread takes the first chunk, and any
// chunk whose thread the system refuses); returns when every chunk is done
template <class F>
void host_parallel(size_t n, size_t grain, const F &f)
{
    const unsigned hw = std::thread::hardware_concurrency();
    const size_t nt = std::min<size_t>(std::min<size_t>(hw ? hw : 1, 16), (n + grain - 1) / std::max<size_t>(grain, 1));
    if (nt <= 1) {
        f((size_t)0, n);
        return;
    }
    const size_t chunk = (n + nt - 1) / nt;
    std::vector<std::thread> th;
    for (size_t t = 1; t < nt; ++t) {
        const size_t b = t * chunk, e = std::min(n, b + chunk);
        if (b >= e) continue;
        try {
            th.emplace_back([&f, b, e] { f(b, e); });
        } catch (...) {
            f(b, e);
        }
    }
    f((size_t)0, std::min(n, chunk));
    for (auto &x : th) x.join();
}

}  // namespace

struct mc_handle {
    int device = 0;
    int precision = MC_PREC_FP32;
    int n_rep = 0;
    int n_sites = 0;
    int n_cells = 0;
    int n_act = 0;
    int stencil_cap = 0;
    size_t smem_bytes = 0;
    int pgrid = 0;                       // blocks of the persistent sweep (0: CUDA graphs instead)
    unsigned int *d_bar = nullptr;       // grid barrier words
    int *d_scan_tot = nullptr;           // per-block scan totals of the persistent sweep
    int wpb = 4;
    double recheck_gap = 1e-5;
    int recompute_every = 0;             // FP64 recompute every k sweeps of sweep_impl (0: off)
    int since_recompute = 0;             // sweeps made since the last one
    double *d_drift = nullptr;           // per replica: last and largest relative drift
    mc_params params{};
    std::vector<RepInfo> reps;
    // page-locked host staging of the state's uploads and downloads, grown on
    // demand (pageable memory when page-locked memory cannot be had)
    void *pin = nullptr;
    size_t pin_bytes = 0;
    std::vector<unsigned char> pageable;
    void *host_buf(size_t bytes)
    {
        if (pin && pin_bytes >= bytes) return pin;
        if (pin) {
            cudaFreeHost(pin);
            pin = nullptr;
            pin_bytes = 0;
        }
        if (cudaHostAlloc(&pin, bytes, cudaHostAllocDefault) == cudaSuccess) {
            pin_bytes = bytes;
            return pin;
        }
        pin = nullptr;
        cudaGetLastError();
        pageable.resize(bytes);
        return pageable.data();
    }
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    int cur = 0;
    bool has_t0 = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    DevState ds{};
    ObsState obs{};
    // multiple-origin correlations (mc_corr_*)
    struct Corr {
        bool on = false;
        std::vector<long long> lags;
        int every = 1;
        long long t = 0;                  // correlation clock: sweeps made by mc_corr_run since the setup
        std::vector<long long> slot_t0;   // origin time per slot, -1: free
        std::vector<void *> bufs;         // device buffers of the setup
        CorrDev dev{};
    } corr;
    // molecular dynamics (mc_md_*)
    struct Md {
        bool on = false;
        MdDev dev{};
        std::vector<double> T, Q;
        std::vector<void *> bufs;
        cudaGraphExec_t graph[2] = {nullptr, nullptr};
    } md;
    std::vector<Buf> allocs;
    // device scratch
    RepInfo *d_rep = nullptr;
    RepParam *d_par = nullptr;
    RepCtr *d_ctr = nullptr;
    ModelDev *d_model = nullptr;
    MixDev *d_mix = nullptr;
    int *d_rep_of_site = nullptr;
    int *d_act_off = nullptr;
    int2 *d_act_slot = nullptr;
    double *d_e_site = nullptr;          // per-cell (or per-site) FP64 partial sums
    double *d_e_out = nullptr;
    long long *d_X = nullptr;
    int *d_types = nullptr;
    double *d_fs = nullptr, *d_fscm = nullptr, *d_c2 = nullptr, *d_q = nullptr, *d_obs_out = nullptr;
    std::vector<RepParam> par_host;
    std::vector<RepParam> par_sent;
    MixDev mix_sent{};
    bool params_valid = false;
    ModelDev model_host{};

    template <class T>
    int alloc(T **p, size_t n)
    {
        void *q = nullptr;
        const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
        if (g_fail_alloc == 0) {
            g_fail_alloc = -1;
            return fail(MC_ERR_CUDA, "cudaMalloc: out of memory (injected by mc_test_fail_alloc)");
        }
        if (g_fail_alloc > 0) --g_fail_alloc;
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) return fail(MC_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        cudaMemset(q, 0, bytes);
        allocs.push_back({q, bytes});
        *p = (T *)q;
        return MC_OK;
    }
};

namespace {

int set_device(const mc_handle *h)
{
    CUDA_TRY(cudaSetDevice(h->device));
    return MC_OK;
}

void default_params(mc_params *p)
{
    p->sigma[0] = 0.9;
    p->sigma[1] = 1.0;
    p->sigma[2] = 1.1;
    p->eps = 1.0;
    p->fene_k = 33.75;
    p->fene_r0 = 1.5;
}

void build_model(const mc_params &p, double gap, ModelDev &md)
{
    std::memset(&md, 0, sizeof md);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const int ab = 3 * a + b;
            const double s = (p.sigma[a] + p.sigma[b]) * 0.5;
            const double s2 = s * s;
            const double R = p.fene_r0 * s;
            md.s2[ab] = s2;
            md.rc2[ab] = kCbrt2 * s2;
            md.R2[ab] = R * R;
            md.s2f[ab] = (float)md.s2[ab];
            md.rc2f[ab] = (float)md.rc2[ab];
            md.R2f[ab] = (float)md.R2[ab];
            md.invR2f[ab] = (float)(1.0 / md.R2[ab]);
        }
    md.eps = p.eps;
    md.e4 = 4.0 * p.eps;
    md.ke = p.fene_k * p.eps;
    md.nke = -md.ke;
    md.epsf = (float)md.eps;
    md.e4f = (float)md.e4;
    md.kef = (float)md.ke;
    md.nkef = (float)md.nke;
    md.bond_guard_f = 0.995f;
    md.recheck_gap_f = (float)gap;
}

// Longest interaction range: the WCA cutoff of any type pair, and the FENE
// divergence of any pair that can form a bond (type pairs inside a molecule's
// multiset, which flips permute but never change).
double interaction_range(const mc_params &p, const int32_t *types, int n_mol)
{
    double smax = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) smax = std::max(smax, 0.5 * (p.sigma[a] + p.sigma[b]));
    double range = std::pow(2.0, 1.0 / 6.0) * smax;
    bool seen[3][3] = {};
    for (int m = 0; m < n_mol; ++m)
        for (int k = 0; k < 3; ++k)
            for (int l = k + 1; l < 3; ++l) seen[types[3 * m + k]][types[3 * m + l]] = true;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (seen[a][b]) range = std::max(range, p.fene_r0 * 0.5 * (p.sigma[a] + p.sigma[b]));
    return range;
}

// smallest cell width in length units for n_c cells per axis
double min_cell_width(double L, int nc)
{
    return std::floor(kTwo32 / nc) * (L / kTwo32);
}

int choose_cells(double L, double range, int request, int *nc_out)
{
    if (L < 2.0 * range) return fail(MC_ERR_INVALID_ARG, "box side smaller than twice the interaction range");
    if (request > 0) {
        if (request % 2 != 0 || request < 2) return fail(MC_ERR_INVALID_ARG, "n_cells must be even and >= 2");
        if (min_cell_width(L, request) < range)
            return fail(MC_ERR_INVALID_ARG, "n_cells makes cells narrower than the interaction range");
        *nc_out = request;
        return MC_OK;
    }
    int nc = 2;
    while (min_cell_width(L, nc + 2) >= range && nc + 2 <= 1024) nc += 2;
    *nc_out = nc;
    return MC_OK;
}

int check_mix(const mc_move_mix *mx)
{
    if (!mx) return fail(MC_ERR_INVALID_ARG, "mix is NULL");
    double s = 0.0;
    for (int k = 0; k < 4; ++k) {
        if (!(mx->p[k] >= 0.0) || !std::isfinite(mx->p[k])) return fail(MC_ERR_INVALID_ARG, "mix probability < 0");
        s += mx->p[k];
    }
    if (std::fabs(s - 1.0) > 1e-9) return fail(MC_ERR_INVALID_ARG, "mix probabilities do not sum to 1");
    if (!(mx->d_atom >= 0.0) || !(mx->d_mol >= 0.0) || !(mx->rot_a >= 0.0) || !std::isfinite(mx->rot_a))
        return fail(MC_ERR_INVALID_ARG, "negative or non-finite step width");
    return MC_OK;
}

// thresholds on a 32-bit word from cumulative probabilities; a threshold past
// which only zero-probability types remain is 2^32
void mix_thresholds(const mc_move_mix *mx, uint64_t thr[3])
{
    double c = 0.0;
    for (int k = 0; k < 3; ++k) {
        c = c + mx->p[k];
        bool tail_zero = true;
        for (int m = k + 1; m < 4; ++m) tail_zero = tail_zero && (mx->p[m] == 0.0);
        const double v = std::floor(c * kTwo32);
        thr[k] = (tail_zero || v >= kTwo32) ? (uint64_t)4294967296ull : (uint64_t)v;
    }
}

int32_t fixed_half_width(double d, double L)
{
    return (int32_t)std::floor(d / L * kTwo32);
}

// Quantise (xyz) or take as given (qfix) and pack the records of all replicas
// (site order) into rec (n_sites entries); validate types, positions and
// bonds.  Host threads take contiguous runs of molecules.  The error reported
// is the one the serial order meets first (replicas in order; within a
// replica every site, in order, before any bond), whichever thread finds it:
// each error has a key (replica, site or bond, index, kind) and the smallest
// key wins.
int pack_records(mc_handle *h, const double *xyz, const uint32_t *qfix, const int32_t *types, int4 *rec)
{
    constexpr uint64_t kNone = ~0ull;
    enum { kType = 0, kFinite = 1 };
    auto site_key = [](int r, int i, int kind) { return ((uint64_t)r << 36) | ((uint64_t)i << 1) | (uint64_t)kind; };
    auto bond_key = [](int r, int m) { return ((uint64_t)r << 36) | (1ull << 35) | ((uint64_t)m << 1); };
    std::atomic<uint64_t> first{kNone};
    const size_t nmol = (size_t)h->n_sites / 3;
    host_parallel(nmol, 8192, [&](size_t mb, size_t me) {
        uint64_t low = kNone;
        int r = (int)(std::upper_bound(h->reps.begin(), h->reps.end(), mb,
                                       [](size_t m, const RepInfo &ri) { return m < (size_t)ri.site_off / 3; }) -
                      h->reps.begin()) - 1;
        for (size_t M = mb; M < me; ++M) {
            while ((size_t)(h->reps[r].site_off + h->reps[r].n_sites) / 3 <= M) ++r;
            const RepInfo &ri = h->reps[r];
            const int m = (int)(M - (size_t)ri.site_off / 3);
            bool ok = true;
            for (int k = 0; k < 3; ++k) {
                const int i = 3 * m + k;
                const size_t g = (size_t)ri.site_off + i;
                const int t = types[g];
                int4 v = make_int4(0, 0, 0, 0);
                uint64_t key = kNone;
                if (t < 0 || t > 2) {
                    key = site_key(r, i, kType);
                } else if (qfix) {
                    v.x = (int)qfix[3 * g + 0];
                    v.y = (int)qfix[3 * g + 1];
                    v.z = (int)qfix[3 * g + 2];
                } else if (!std::isfinite(xyz[3 * g + 0]) || !std::isfinite(xyz[3 * g + 1]) ||
                           !std::isfinite(xyz[3 * g + 2])) {
                    key = site_key(r, i, kFinite);
                } else {
                    v.x = (int)quantize(xyz[3 * g + 0], ri.L);
                    v.y = (int)quantize(xyz[3 * g + 1], ri.L);
                    v.z = (int)quantize(xyz[3 * g + 2], ri.L);
                }
                v.w = (m << 4) | (k << 2) | (t & 3);
                rec[g] = v;
                if (key != kNone) {
                    ok = false;
                    low = std::min<uint64_t>(low, key);
                }
            }
            if (!ok) continue;
            // every bond strictly inside its FENE range
            for (int k = 0; k < 3; ++k)
                for (int l = k + 1; l < 3; ++l) {
                    const int4 a = rec[ri.site_off + 3 * m + k], b = rec[ri.site_off + 3 * m + l];
                    double r2 = 0.0;
                    const int da[3] = {(int)((uint32_t)b.x - (uint32_t)a.x), (int)((uint32_t)b.y - (uint32_t)a.y),
                                       (int)((uint32_t)b.z - (uint32_t)a.z)};
                    for (int ax = 0; ax < 3; ++ax) {
                        const double x = (double)da[ax] * ri.h;
                        r2 += x * x;
                    }
                    if (!(r2 < h->model_host.R2[3 * (a.w & 3) + (b.w & 3)])) low = std::min<uint64_t>(low, bond_key(r, m));
                }
        }
        uint64_t cur = first.load();
        while (low < cur && !first.compare_exchange_weak(cur, low)) {
        }
    });
    const uint64_t key = first.load();
    if (key == kNone) return MC_OK;
    const int r = (int)(key >> 36);
    if ((key >> 35) & 1)
        return fail(MC_ERR_BAD_STATE, "a bond is at or beyond its FENE range (replica " + std::to_string(r) +
                                          ", molecule " + std::to_string((int)((key >> 1) & 0x3FFFFFFFull)) + ")");
    if ((key & 1) == kType) return fail(MC_ERR_INVALID_ARG, "type outside {0,1,2}");
    return fail(MC_ERR_BAD_STATE, "non-finite position");
}

int check_device_errors(mc_handle *h)
{
    int e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, h->ds.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (e & ERR_STENCIL) return fail(MC_ERR_CELL_OVERFLOW, "a cell neighbourhood exceeded the staging capacity");
    if (e & ERR_TERMS) return fail(MC_ERR_CELL_OVERFLOW, "too many nonzero FP64 terms in one move");
    if (e & ERR_TIMEOUT) return fail(MC_ERR_TIMEOUT, "a device wait timed out");
    return MC_OK;
}

// energy of each replica into h->d_e_out (device)
int enqueue_energy(mc_handle *h)
{
    launch_energy(h->ds, h->cur, h->d_e_site, h->d_e_out, h->stream);
    CUDA_TRY(cudaGetLastError());
    return MC_OK;
}

int rebuild_and_reset(mc_handle *h, const int4 *rec, const std::vector<int> *img = nullptr)
{
    // upload in site order into the spare buffer, sort into the other
    const int spare = h->cur;
    CUDA_TRY(cudaMemcpyAsync(h->ds.rec[spare], rec, sizeof(int4) * (size_t)h->n_sites, cudaMemcpyHostToDevice,
                             h->stream));
    launch_cell_list(h->ds, spare, spare ^ 1, h->stream);
    h->cur = spare ^ 1;
    if (img)
        CUDA_TRY(cudaMemcpyAsync(h->ds.img, img->data(), sizeof(int) * img->size(), cudaMemcpyHostToDevice, h->stream));
    else
        CUDA_TRY(cudaMemsetAsync(h->ds.img, 0, sizeof(int) * 3 * (size_t)h->n_sites, h->stream));
    int rc = enqueue_energy(h);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(h->ds.e_run, h->d_e_out, sizeof(double) * h->n_rep, cudaMemcpyDeviceToDevice, h->stream));
    std::vector<double> e(h->n_rep);
    CUDA_TRY(cudaMemcpyAsync(e.data(), h->d_e_out, sizeof(double) * h->n_rep, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    rc = check_device_errors(h);
    if (rc) return rc;
    for (int r = 0; r < h->n_rep; ++r)
        if (!std::isfinite(e[r])) return fail(MC_ERR_BAD_STATE, "non-finite energy in replica " + std::to_string(r));
    h->has_t0 = false;
    return MC_OK;
}

int upload_params(mc_handle *h, const double *T, const mc_move_mix *mix, const uint64_t *seeds, bool same_T_seed)
{
    for (int r = 0; r < h->n_rep; ++r) {
        const double t = same_T_seed ? T[0] : T[r];
        if (!(t > 0.0) || !std::isfinite(t)) return fail(MC_ERR_INVALID_ARG, "temperature must be positive");
        RepParam &p = h->par_host[r];
        p.T = t;
        p.T32 = (float)t;
        p.pad = 0;
        p.seed = same_T_seed ? seeds[0] : seeds[r];
        p.D_atom = fixed_half_width(mix->d_atom, h->reps[r].L);
        p.D_mol = fixed_half_width(mix->d_mol, h->reps[r].L);
        if (p.D_atom < 0 || p.D_mol < 0 || (double)p.D_atom > 0.25 * kTwo32 || (double)p.D_mol > 0.25 * kTwo32)
            return fail(MC_ERR_INVALID_ARG, "step width out of range");
    }
    MixDev mx{};
    mix_thresholds(mix, mx.thr);
    mx.rot_a = mix->rot_a;
    // identical parameters are not uploaded again, so that consecutive calls
    // stay asynchronous (a copy from pageable memory waits for the stream)
    if (h->params_valid && std::memcmp(h->par_sent.data(), h->par_host.data(), sizeof(RepParam) * h->n_rep) == 0 &&
        std::memcmp(&h->mix_sent, &mx, sizeof(MixDev)) == 0)
        return MC_OK;
    CUDA_TRY(cudaMemcpyAsync(h->d_par, h->par_host.data(), sizeof(RepParam) * h->n_rep, cudaMemcpyHostToDevice,
                             h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->d_mix, &mx, sizeof(MixDev), cudaMemcpyHostToDevice, h->stream));
    h->par_sent = h->par_host;
    h->mix_sent = mx;
    h->params_valid = true;
    return MC_OK;
}

int ensure_graph(mc_handle *h, int buf)
{
    if (h->graph[buf]) return MC_OK;
    cudaStream_t cs;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    launch_cell_list(h->ds, buf, buf ^ 1, cs);
    LogArgs none{nullptr, 0, 0};
    launch_phases(h->ds, buf ^ 1, h->wpb, none, cs);
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(MC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&h->graph[buf], g, 0);
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return fail(MC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return MC_OK;
}

int create_impl(mc_handle **out, int n_rep, const double *L, const int32_t *n_mol, const double *xyz,
                const int32_t *types, const mc_params *params, const mc_options *opts)
{
    if (!out) return fail(MC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_rep < 1 || !L || !n_mol || !xyz || !types) return fail(MC_ERR_INVALID_ARG, "NULL input or n_rep < 1");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return fail(MC_ERR_NO_DEVICE, "no CUDA device");
    mc_options o{};
    o.precision = MC_PREC_FP32;
    if (opts) o = *opts;
    if (o.precision != MC_PREC_FP32 && o.precision != MC_PREC_FP64) return fail(MC_ERR_INVALID_ARG, "precision");
    if (o.device < 0 || o.device >= ndev) return fail(MC_ERR_INVALID_ARG, "device ordinal");
    if (o.recompute_every < 0) return fail(MC_ERR_INVALID_ARG, "recompute_every < 0");
    if (o.wait_limit_log2 < 0 || o.wait_limit_log2 > 30) return fail(MC_ERR_INVALID_ARG, "wait_limit_log2");
    mc_params p;
    default_params(&p);
    if (params) p = *params;
    for (int k = 0; k < 3; ++k)
        if (!(p.sigma[k] > 0.0)) return fail(MC_ERR_INVALID_ARG, "sigma must be positive");
    if (!(p.eps > 0.0) || !(p.fene_k >= 0.0) || !(p.fene_r0 > 0.0)) return fail(MC_ERR_INVALID_ARG, "potential params");

    auto *h = new mc_handle();
    h->device = o.device;
    h->precision = o.precision;
    h->params = p;
    h->recheck_gap = o.recheck_gap > 0.0 ? o.recheck_gap : 1e-5;
    h->recompute_every = o.recompute_every;
    h->n_rep = n_rep;
    build_model(p, h->recheck_gap, h->model_host);

    // layout
    long long sites = 0, cells = 0, act = 0;
    double max_stencil = 0.0;
    std::vector<int> act_off(n_rep + 1, 0), rep_of_site;
    std::vector<double> cell_load(n_rep, 0.0);
    for (int r = 0; r < n_rep; ++r) {
        if (n_mol[r] < 1 || n_mol[r] > kMaxMolecules) {
            delete h;
            return fail(MC_ERR_INVALID_ARG, "n_mol outside [1, 2^27 - 2]");
        }
        if (!(L[r] > 0.0) || !std::isfinite(L[r])) {
            delete h;
            return fail(MC_ERR_INVALID_ARG, "box side must be positive");
        }
        const int32_t *tr = types + sites;
        for (long long i = 0; i < 3LL * n_mol[r]; ++i)
            if (tr[i] < 0 || tr[i] > 2) {
                delete h;
                return fail(MC_ERR_INVALID_ARG, "type outside {0,1,2}");
            }
        const double range = interaction_range(p, tr, n_mol[r]);
        int nc = 0;
        int rc = choose_cells(L[r], range, o.n_cells, &nc);
        if (rc) {
            delete h;
            return rc;
        }
        RepInfo ri{};
        ri.n_sites = 3 * n_mol[r];
        ri.site_off = (int)sites;
        ri.nc = nc;
        ri.cell_off = (int)cells;
        ri.act_off = (int)act;
        ri.L = L[r];
        ri.h = L[r] / kTwo32;
        ri.inv_h = kTwo32 / L[r];
        ri.hf = (float)ri.h;
        ri.h2f = (float)(ri.h * ri.h);
        // the radii of the screens and of the conflict test, in FP32 as the
        // kernels use them (one rounding per operation)
        float rc2max = 0.f;
        for (int k = 0; k < 9; ++k) rc2max = std::fmax(rc2max, h->model_host.rc2f[k]);
        ri.pre_r2 = rc2max * 1.01f;
        ri.r2q = ri.pre_r2 / ri.h2f;
        ri.rconf = rc2max * 1.0201f / ri.h2f;
        h->reps.push_back(ri);
        for (int i = 0; i < ri.n_sites; ++i) rep_of_site.push_back(r);
        sites += ri.n_sites;
        cells += (long long)nc * nc * nc;
        act += (long long)(nc / 2) * (nc / 2) * (nc / 2);
        act_off[r + 1] = (int)act;
        cell_load[r] = (double)ri.n_sites / ((double)nc * nc * nc);
        // neighbourhood size: mean plus six standard deviations
        // (counts are at most Poisson-distributed in a liquid) and a margin
        const double per_cell = (double)ri.n_sites / ((double)nc * nc * nc);
        const double mean_nb = 27.0 * per_cell;
        const double st = (nc == 2) ? (double)ri.n_sites : mean_nb + 6.0 * std::sqrt(mean_nb) + 32.0;
        max_stencil = std::max(max_stencil, std::min(st, (double)ri.n_sites));
        if (sites > (1LL << 30)) {
            delete h;
            return fail(MC_ERR_INVALID_ARG, "too many sites");
        }
    }
    h->n_sites = (int)sites;
    h->n_cells = (int)cells;
    h->n_act = (int)act;
    // active-cell slots in schedule order: replicas with the most atoms per
    // cell first (a cell's phase costs about its atoms times its neighbourhood,
    // so the dense replicas' cells go in the first waves of a phase launch and
    // the light ones fill its tail); within a replica, active-cell order
    std::vector<int2> act_slot;
    if (n_rep > 1) {
        std::vector<int> order(n_rep);
        for (int r = 0; r < n_rep; ++r) order[r] = r;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cell_load[a] > cell_load[b]; });
        act_slot.reserve((size_t)act);
        for (int r : order)
            for (int a = 0; a < act_off[r + 1] - act_off[r]; ++a) act_slot.push_back(make_int2(r, a));
    }
    // staging capacity: the neighbourhood (mean + 6 sigma + 32) plus the padding records, a multiple of 32
    int cap = o.stencil_cap > 0 ? o.stencil_cap : ((int)std::ceil(max_stencil) + kPadSlots + 31) / 32 * 32;
    h->stencil_cap = cap;
    // warps per cell: spread small grids over more warps so that every SM has
    // work; large grids keep one warp per cell (enough cells to fill the GPU)
    if (o.warps_per_cell != 0 && o.warps_per_cell != 1 && o.warps_per_cell != 2 && o.warps_per_cell != 4 &&
        o.warps_per_cell != 8) {
        delete h;
        return fail(MC_ERR_INVALID_ARG, "warps_per_cell must be 0, 1, 2, 4 or 8");
    }
    if (o.warps_per_cell > 0) h->wpb = o.warps_per_cell;
    else h->wpb = h->n_act >= 152 * 12 ? 1 : (h->n_act >= 152 * 3 ? 2 : 4);
    h->smem_bytes = phase_smem_bytes(cap, h->wpb);
    if (h->smem_bytes > 220u * 1024u) {
        delete h;
        return fail(MC_ERR_INVALID_ARG, "stencil capacity too large for shared memory");
    }

    int rc = set_device(h);
    if (rc) {
        delete h;
        return rc;
    }
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        return fail(MC_ERR_CUDA, "stream create");
    }
    h->stream = h->own_stream;

    DevState &d = h->ds;
    d.n_rep = n_rep;
    d.n_sites = h->n_sites;
    d.n_cells = h->n_cells;
    d.n_act = h->n_act;
    d.stencil_cap = cap;
    d.precision = h->precision;
    d.wait_limit = o.wait_limit_log2 > 0 ? (1u << o.wait_limit_log2) : 0u;
    const int M_tot = h->n_sites / 3;
    int4 *r0, *r1;
    int *cc, *cs, *co, *so, *img, *err;
    double *cde, *erun;
    unsigned long long *stats;
    if ((rc = h->alloc(&h->d_rep, n_rep)) || (rc = h->alloc(&h->d_par, n_rep)) || (rc = h->alloc(&h->d_ctr, n_rep)) ||
        (rc = h->alloc(&h->d_model, 1)) || (rc = h->alloc(&h->d_mix, 1)) ||
        (rc = h->alloc(&h->d_rep_of_site, h->n_sites)) || (rc = h->alloc(&h->d_act_off, n_rep + 1)) ||
        (rc = h->alloc(&h->d_act_slot, n_rep > 1 ? h->n_act : 0)) ||
        (rc = h->alloc(&r0, h->n_sites)) || (rc = h->alloc(&r1, h->n_sites)) || (rc = h->alloc(&cc, h->n_cells)) ||
        (rc = h->alloc(&cs, h->n_cells + 1)) || (rc = h->alloc(&co, h->n_sites)) || (rc = h->alloc(&so, h->n_sites)) ||
        (rc = h->alloc(&img, 3 * (size_t)h->n_sites)) || (rc = h->alloc(&cde, h->n_cells)) ||
        (rc = h->alloc(&stats, (size_t)STAT_N * n_rep)) || (rc = h->alloc(&erun, n_rep)) ||
        (rc = h->alloc(&err, 1)) || (rc = h->alloc(&h->d_e_site, std::max(h->n_sites, h->n_cells))) ||
        (rc = h->alloc(&h->d_e_out, n_rep)) || (rc = h->alloc(&h->d_X, 3 * (size_t)h->n_sites)) ||
        (rc = h->alloc(&h->d_types, h->n_sites)) || (rc = h->alloc(&h->obs.X0, 3 * (size_t)h->n_sites)) ||
        (rc = h->alloc(&h->obs.kref, M_tot)) || (rc = h->alloc(&h->obs.u0, 3 * (size_t)M_tot)) ||
        (rc = h->alloc(&h->d_fs, h->n_sites)) || (rc = h->alloc(&h->d_fscm, M_tot)) ||
        (rc = h->alloc(&h->d_c2, M_tot)) || (rc = h->alloc(&h->d_q, 6 * 256)) ||
        (rc = h->alloc(&h->d_obs_out, 3 * (size_t)n_rep)) ||
        (rc = h->alloc(&h->ds.att_rnd, 2 * (size_t)h->n_sites)) || (rc = h->alloc(&h->d_bar, 2)) ||
        (rc = h->alloc(&h->ds.cell_done, h->n_cells)) || (rc = h->alloc(&h->ds.cell_count2, h->n_cells)) ||
        (rc = h->alloc(&h->d_scan_tot, kMaxPersistentBlocks)) ||
        (rc = h->alloc(&h->ds.scan_part, (size_t)h->n_cells / 1024 + 2)) || (rc = h->alloc(&h->d_drift, 2 * (size_t)n_rep)) ||
        (rc = h->precision == MC_PREC_FP64 ? h->alloc(&h->ds.att_thr64, h->n_sites)
                                           : h->alloc(&h->ds.att_thr32, h->n_sites))) {
        mc_destroy(h);
        return rc;
    }
    d.rep = h->d_rep;
    d.par = h->d_par;
    d.ctr = h->d_ctr;
    d.model = h->d_model;
    d.mix = h->d_mix;
    d.rep_of_site = h->d_rep_of_site;
    d.act_off = h->d_act_off;
    d.act_slot = n_rep > 1 ? h->d_act_slot : nullptr;
    d.rec[0] = r0;
    d.rec[1] = r1;
    d.cell_count = cc;
    d.cell_start = cs;
    d.cell_of = co;
    d.slot_of = so;
    d.img = img;
    d.cell_dE = cde;
    d.stats = stats;
    d.e_run = erun;
    d.err = err;

    h->par_host.assign(n_rep, RepParam{1.0, 0, 0, 0});
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!up(h->d_rep, h->reps.data(), sizeof(RepInfo) * n_rep) || !up(h->d_model, &h->model_host, sizeof(ModelDev)) ||
        !up(h->d_rep_of_site, rep_of_site.data(), sizeof(int) * h->n_sites) ||
        !up(h->d_act_off, act_off.data(), sizeof(int) * (n_rep + 1)) ||
        (n_rep > 1 && !up(h->d_act_slot, act_slot.data(), sizeof(int2) * h->n_act)) ||
        !up(h->d_par, h->par_host.data(), sizeof(RepParam) * n_rep)) {
        mc_destroy(h);
        return fail(MC_ERR_CUDA, "upload of tables failed");
    }
    if (phase_set_smem_limit((int)h->smem_bytes) != 0) {
        mc_destroy(h);
        return fail(MC_ERR_CUDA, "cannot reserve shared memory for the sweep kernel");
    }
    // sweeps run as one persistent cooperative launch per call unless graphs are asked for
    if (o.launch_mode != 1) h->pgrid = persistent_grid(h->ds, h->wpb, kMaxPersistentBlocks);
    if (o.launch_mode == 2 && h->pgrid == 0) {
        mc_destroy(h);
        return fail(MC_ERR_INVALID_ARG, "persistent sweeps need cooperative launch support");
    }
    int4 *rec = (int4 *)h->host_buf(sizeof(int4) * (size_t)h->n_sites);
    rc = pack_records(h, xyz, nullptr, types, rec);
    if (rc == MC_OK) rc = rebuild_and_reset(h, rec);
    if (rc) {
        std::string msg = g_err;
        mc_destroy(h);
        return fail(rc, msg);
    }
    *out = h;
    return MC_OK;
}

}  // namespace

extern "C" {

int mc_create(mc_handle **out, double L, int n_mol, const double *xyz, const int32_t *types, const mc_params *params,
              const mc_options *opts)
{
    const int32_t nm = n_mol;
    return create_impl(out, 1, &L, &nm, xyz, types, params, opts);
}

int mc_create_batch(mc_handle **out, int n_rep, const double *L, const int32_t *n_mol, const double *xyz,
                    const int32_t *types, const mc_params *params, const mc_options *opts)
{
    return create_impl(out, n_rep, L, n_mol, xyz, types, params, opts);
}

// Release the buffers of a correlation setup (after the stream is idle).
static void corr_free(mc_handle *h)
{
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void *b : h->corr.bufs) cudaFree(b);
    h->corr = mc_handle::Corr{};
}

// Release the buffers and graphs of an MD setup (after the stream is idle).
static void md_free(mc_handle *h)
{
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int b = 0; b < 2; ++b)
        if (h->md.graph[b]) cudaGraphExecDestroy(h->md.graph[b]);
    for (void *b : h->md.bufs) cudaFree(b);
    h->md = mc_handle::Md{};
}

void mc_destroy(mc_handle *h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    corr_free(h);
    md_free(h);
    for (int b = 0; b < 2; ++b)
        if (h->graph[b]) cudaGraphExecDestroy(h->graph[b]);
    for (auto &a : h->allocs) cudaFree(a.p);
    if (h->pin) cudaFreeHost(h->pin);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

int mc_set_stream(mc_handle *h, void *stream)
{
    if (!h) return fail(MC_ERR_INVALID_ARG, "NULL handle");
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    return MC_OK;
}

static int sweep_impl(mc_handle *h, int n_sweeps, const double *T, const mc_move_mix *mix, const uint64_t *seeds,
                      bool same)
{
    if (!h) return fail(MC_ERR_INVALID_ARG, "NULL handle");
    if (n_sweeps < 0) return fail(MC_ERR_INVALID_ARG, "n_sweeps < 0");
    if (!T || !seeds) return fail(MC_ERR_INVALID_ARG, "NULL T or seeds");
    int rc = check_mix(mix);
    if (rc) return rc;
    if ((rc = set_device(h))) return rc;
    if ((rc = upload_params(h, T, mix, seeds, same))) return rc;
    while (n_sweeps > 0) {
        // the sweeps up to the next periodic FP64 recompute (all of them when off)
        const int chunk =
            h->recompute_every > 0 ? std::min(n_sweeps, h->recompute_every - h->since_recompute) : n_sweeps;
        if (h->pgrid > 0) {
            // all sweeps of the chunk in one cooperative launch (which expects
            // zero counts in cell_count on entry and clears cell_count2 itself)
            CUDA_TRY(cudaMemsetAsync(h->ds.cell_count, 0, sizeof(int) * h->n_cells, h->stream));
            CUDA_TRY(cudaMemsetAsync(h->d_bar, 0, sizeof(unsigned int) * 2, h->stream));
            CUDA_TRY(cudaMemsetAsync(h->ds.cell_done, 0, sizeof(unsigned int) * h->n_cells, h->stream));
            const int e = launch_persistent(h->ds, h->cur, chunk, h->wpb, h->pgrid, h->d_bar, h->d_scan_tot, h->stream);
            if (e != 0)
                return fail(MC_ERR_CUDA, std::string("persistent sweep launch: ") + cudaGetErrorString((cudaError_t)e));
            h->cur ^= (chunk & 1);
        } else {
            for (int s = 0; s < chunk; ++s) {
                if ((rc = ensure_graph(h, h->cur))) return rc;
                CUDA_TRY(cudaGraphLaunch(h->graph[h->cur], h->stream));
                h->cur ^= 1;
            }
        }
        n_sweeps -= chunk;
        if (h->recompute_every > 0 && (h->since_recompute += chunk) >= h->recompute_every) {
            // FP64 total from the state, drift of the running total, restart from it
            if ((rc = enqueue_energy(h))) return rc;
            launch_drift(h->ds, h->d_e_out, h->d_drift, h->stream);
            h->since_recompute = 0;
        }
    }
    CUDA_TRY(cudaGetLastError());
    return MC_OK;
}

int mc_sweep(mc_handle *h, int n_sweeps, double T, const mc_move_mix *mix, uint64_t seed)
{
    return sweep_impl(h, n_sweeps, &T, mix, &seed, true);
}

int mc_sweep_batch(mc_handle *h, int n_sweeps, const double *T, const mc_move_mix *mix, const uint64_t *seeds)
{
    return sweep_impl(h, n_sweeps, T, mix, seeds, false);
}

int mc_sweep_logged(mc_handle *h, int n_sweeps, const double *T, const mc_move_mix *mix, const uint64_t *seeds,
                    mc_log_entry *log_out)
{
    if (!h || !log_out) return fail(MC_ERR_INVALID_ARG, "NULL handle or log");
    if (n_sweeps < 0 || !T || !seeds) return fail(MC_ERR_INVALID_ARG, "bad arguments");
    int rc = check_mix(mix);
    if (rc) return rc;
    if ((rc = set_device(h))) return rc;
    if ((rc = upload_params(h, T, mix, seeds, false))) return rc;
    if (n_sweeps == 0) return MC_OK;
    uint64_t sweep0 = 0;
    CUDA_TRY(cudaMemcpy(&sweep0, &h->d_ctr[0].sweep, sizeof(uint64_t), cudaMemcpyDeviceToHost));
    const size_t n = (size_t)n_sweeps * (size_t)h->n_sites;
    mc_log_entry *dlog = nullptr;
    CUDA_TRY(cudaMalloc(&dlog, sizeof(mc_log_entry) * n));
    cudaMemsetAsync(dlog, 0xff, sizeof(mc_log_entry) * n, h->stream);
    LogArgs lg{dlog, n_sweeps, sweep0};
    for (int s = 0; s < n_sweeps; ++s) {
        launch_cell_list(h->ds, h->cur, h->cur ^ 1, h->stream);
        launch_phases(h->ds, h->cur ^ 1, h->wpb, lg, h->stream);
        h->cur ^= 1;
    }
    cudaError_t e = cudaMemcpyAsync(log_out, dlog, sizeof(mc_log_entry) * n, cudaMemcpyDeviceToHost, h->stream);
    cudaError_t e2 = cudaStreamSynchronize(h->stream);
    cudaFree(dlog);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(MC_ERR_CUDA, std::string("logged sweep: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    return check_device_errors(h);
}

int mc_sweep_timed(mc_handle *h, int n_sweeps, const double *T, const mc_move_mix *mix, const uint64_t *seeds,
                   double *ms_out)
{
    if (!h || !ms_out || !T || !seeds || n_sweeps < 0) return fail(MC_ERR_INVALID_ARG, "bad arguments");
    int rc = check_mix(mix);
    if (rc) return rc;
    if ((rc = set_device(h))) return rc;
    if ((rc = upload_params(h, T, mix, seeds, false))) return rc;
    cudaEvent_t ev[4];
    for (auto &e : ev) CUDA_TRY(cudaEventCreate(&e));
    double tot[3] = {0.0, 0.0, 0.0};
    LogArgs none{nullptr, 0, 0};
    for (int s = 0; s < n_sweeps; ++s) {
        cudaEventRecord(ev[0], h->stream);
        launch_cell_list(h->ds, h->cur, h->cur ^ 1, h->stream);
        cudaEventRecord(ev[1], h->stream);
        launch_colour_phases(h->ds, h->cur ^ 1, h->wpb, none, h->stream);
        cudaEventRecord(ev[2], h->stream);
        launch_finalize(h->ds, h->stream);
        cudaEventRecord(ev[3], h->stream);
        h->cur ^= 1;
        cudaError_t e = cudaEventSynchronize(ev[3]);
        if (e != cudaSuccess) {
            for (auto &x : ev) cudaEventDestroy(x);
            return fail(MC_ERR_CUDA, std::string("timed sweep: ") + cudaGetErrorString(e));
        }
        for (int k = 0; k < 3; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            tot[k] += ms;
        }
    }
    for (auto &x : ev) cudaEventDestroy(x);
    for (int k = 0; k < 3; ++k) ms_out[k] = tot[k];
    return check_device_errors(h);
}

// Switch the cell schedule: warps per cell W and the launch form.
static int set_schedule(mc_handle *h, int W, bool persistent)
{
    const size_t sm = phase_smem_bytes(h->stencil_cap, W);
    if (sm > 220u * 1024u) return MC_ERR_INVALID_ARG;
    if (phase_set_smem_limit((int)sm) != 0) return MC_ERR_CUDA;
    if (W != h->wpb)
        for (int b = 0; b < 2; ++b)
            if (h->graph[b]) {
                cudaGraphExecDestroy(h->graph[b]);
                h->graph[b] = nullptr;
            }
    h->wpb = W;
    h->smem_bytes = sm;
    h->pgrid = persistent ? persistent_grid(h->ds, W, kMaxPersistentBlocks) : 0;
    return (persistent && h->pgrid == 0) ? MC_ERR_INVALID_ARG : MC_OK;
}

int mc_autotune(mc_handle *h, int n_sweeps, const double *T, const mc_move_mix *mix, const uint64_t *seeds,
                double *results)
{
    if (!h || !T || !seeds || n_sweeps < 1) return fail(MC_ERR_INVALID_ARG, "bad arguments");
    int rc = check_mix(mix);
    if (rc) return rc;
    if ((rc = set_device(h))) return rc;
    // device snapshot of everything a sweep changes
    const size_t n = (size_t)h->n_sites, R = (size_t)h->n_rep;
    const size_t b_rec = sizeof(int4) * n, b_img = sizeof(int) * 3 * n, b_e = sizeof(double) * R,
                 b_st = sizeof(unsigned long long) * STAT_N * R, b_ct = sizeof(RepCtr) * R;
    unsigned char *snap = nullptr;
    CUDA_TRY(cudaMalloc(&snap, b_rec + b_img + b_e + b_st + b_ct));
    const int cur0 = h->cur, W0 = h->wpb;
    const bool p0 = h->pgrid > 0;
    auto copy_all = [&](bool save) {
        void *dev[5] = {h->ds.rec[cur0], h->ds.img, h->ds.e_run, h->ds.stats, h->ds.ctr};
        const size_t sz[5] = {b_rec, b_img, b_e, b_st, b_ct};
        size_t off = 0;
        for (int k = 0; k < 5; ++k) {
            if (save) cudaMemcpyAsync(snap + off, dev[k], sz[k], cudaMemcpyDeviceToDevice, h->stream);
            else cudaMemcpyAsync(dev[k], snap + off, sz[k], cudaMemcpyDeviceToDevice, h->stream);
            off += sz[k];
        }
        h->cur = cur0;
    };
    copy_all(true);
    // the trial sweeps make no periodic recompute (the drift figures and the
    // recompute count stay as they are)
    const int every0 = h->recompute_every, since0 = h->since_recompute;
    h->recompute_every = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int Ws[4] = {1, 2, 4, 8};
    double best = 1e300;
    int bestW = W0;
    bool bestP = p0;
    for (int form = 0; form < 2; ++form) {
        for (int k = 0; k < 4; ++k) {
            double ms = -1.0;
            if (set_schedule(h, Ws[k], form == 0) == MC_OK) {
                copy_all(false);
                rc = sweep_impl(h, 1, T, mix, seeds, false);   // first use: graph capture, caches
                if (rc == MC_OK) {
                    copy_all(false);
                    cudaEventRecord(e0, h->stream);
                    rc = sweep_impl(h, n_sweeps, T, mix, seeds, false);
                    cudaEventRecord(e1, h->stream);
                }
                if (rc == MC_OK && cudaEventSynchronize(e1) == cudaSuccess) {
                    float f = 0.f;
                    cudaEventElapsedTime(&f, e0, e1);
                    ms = f / n_sweeps;
                    if (ms < best) {
                        best = ms;
                        bestW = Ws[k];
                        bestP = form == 0;
                    }
                }
            }
            if (results) results[4 * form + k] = ms;
        }
    }
    copy_all(false);
    h->recompute_every = every0;
    h->since_recompute = since0;
    rc = set_schedule(h, bestW, bestP);
    cudaStreamSynchronize(h->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(snap);
    if (rc) return fail(rc, "autotune: cannot restore the chosen schedule");
    return check_device_errors(h);
}

int mc_energy_device(mc_handle *h, double *dev_E_out)
{
    if (!h || !dev_E_out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    int rc = set_device(h);
    if (rc) return rc;
    if ((rc = enqueue_energy(h))) return rc;
    CUDA_TRY(cudaMemcpyAsync(dev_E_out, h->d_e_out, sizeof(double) * h->n_rep, cudaMemcpyDeviceToDevice, h->stream));
    return MC_OK;
}

int mc_sync(mc_handle *h)
{
    if (!h) return fail(MC_ERR_INVALID_ARG, "NULL handle");
    int rc = set_device(h);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    CUDA_TRY(cudaGetLastError());
    return check_device_errors(h);
}

int mc_energy(mc_handle *h, double *E_out)
{
    if (!h || !E_out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    int rc = set_device(h);
    if (rc) return rc;
    if ((rc = enqueue_energy(h))) return rc;
    CUDA_TRY(cudaMemcpyAsync(E_out, h->d_e_out, sizeof(double) * h->n_rep, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return check_device_errors(h);
}

int mc_pressure(mc_handle *h, const double *T, double *out)
{
    if (!h || !T || !out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    for (int r = 0; r < h->n_rep; ++r)
        if (!(T[r] > 0.0) || !std::isfinite(T[r])) return fail(MC_ERR_INVALID_ARG, "temperature must be positive");
    int rc = set_device(h);
    if (rc) return rc;
    launch_virial(h->ds, h->cur, h->d_e_site, h->d_e_out, h->stream);
    CUDA_TRY(cudaGetLastError());
    std::vector<double> w(h->n_rep);
    CUDA_TRY(cudaMemcpyAsync(w.data(), h->d_e_out, sizeof(double) * h->n_rep, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int r = 0; r < h->n_rep; ++r) {
        const double V = h->reps[r].L * h->reps[r].L * h->reps[r].L;
        out[2 * r] = w[r];
        out[2 * r + 1] = (double)h->reps[r].n_sites * T[r] / V + w[r] / (3.0 * V);
    }
    return check_device_errors(h);
}

int mc_cell_grid(double L, int n_mol, const int32_t *types, const mc_params *params, int request, int *nc_out,
                 double *range_out)
{
    if (!types || !nc_out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    if (n_mol < 1 || n_mol > kMaxMolecules) return fail(MC_ERR_INVALID_ARG, "n_mol outside [1, 2^27 - 2]");
    if (!(L > 0.0) || !std::isfinite(L)) return fail(MC_ERR_INVALID_ARG, "box side must be positive");
    for (long long i = 0; i < 3LL * n_mol; ++i)
        if (types[i] < 0 || types[i] > 2) return fail(MC_ERR_INVALID_ARG, "type outside {0,1,2}");
    mc_params p;
    default_params(&p);
    if (params) p = *params;
    const double range = interaction_range(p, types, n_mol);
    if (range_out) *range_out = range;
    return choose_cells(L, range, request, nc_out);
}

int mc_structure_factor(mc_handle *h, const double *qvec, int n_q, double *out)
{
    if (!h || !qvec || !out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    if (n_q < 1 || n_q > 65535) return fail(MC_ERR_INVALID_ARG, "1 <= n_q <= 65535");
    int rc = set_device(h);
    if (rc) return rc;
    double *dq = nullptr, *dout = nullptr;
    CUDA_TRY(cudaMallocAsync(&dq, sizeof(double) * 3 * n_q, h->stream));
    cudaError_t e = cudaMallocAsync(&dout, sizeof(double) * (size_t)n_q * h->n_rep, h->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(dq, h->stream);
        return fail(MC_ERR_CUDA, std::string("structure factor: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(dq, qvec, sizeof(double) * 3 * n_q, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        launch_gather(h->ds, h->cur, h->d_X, h->d_types, h->stream);
        launch_sq(h->ds, h->d_X, dq, n_q, dout, h->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, dout, sizeof(double) * (size_t)n_q * h->n_rep, cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(dq, h->stream);
    cudaFreeAsync(dout, h->stream);
    const cudaError_t e2 = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(MC_ERR_CUDA, std::string("structure factor: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    return check_device_errors(h);
}

int mc_pair_histogram(mc_handle *h, double dr, int n_bins, uint64_t *counts, double *g)
{
    if (!h || !counts) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    if (!(dr > 0.0) || !std::isfinite(dr) || n_bins < 1 || n_bins > 4096)
        return fail(MC_ERR_INVALID_ARG, "dr > 0 and 1 <= n_bins <= 4096");
    int max_sites = 0;
    for (auto &r : h->reps) {
        if (dr * n_bins > 0.5 * r.L) return fail(MC_ERR_INVALID_ARG, "n_bins * dr exceeds half a box side");
        max_sites = std::max(max_sites, r.n_sites);
    }
    int rc = set_device(h);
    if (rc) return rc;
    const size_t n = (size_t)n_bins * h->n_rep;
    unsigned long long *dc = nullptr;
    CUDA_TRY(cudaMallocAsync(&dc, sizeof(unsigned long long) * n, h->stream));
    cudaError_t e = cudaMemsetAsync(dc, 0, sizeof(unsigned long long) * n, h->stream);
    if (e == cudaSuccess) {
        launch_gather(h->ds, h->cur, h->d_X, h->d_types, h->stream);
        launch_pair_hist(h->ds, h->d_X, max_sites, dr, n_bins, dc, h->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(counts, dc, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(dc, h->stream);
    const cudaError_t e2 = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(MC_ERR_CUDA, std::string("pair histogram: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    if (g) {
        // g(r) at the bin centres: 2 counts / (N rho shell volume), rho = N / V
        const double pi = 3.14159265358979323846;
        for (int r = 0; r < h->n_rep; ++r) {
            const double N = (double)h->reps[r].n_sites, V = h->reps[r].L * h->reps[r].L * h->reps[r].L;
            for (int b = 0; b < n_bins; ++b) {
                const double r0 = b * dr, r1 = (b + 1) * dr;
                const double shell = 4.0 / 3.0 * pi * (r1 * r1 * r1 - r0 * r0 * r0);
                g[(size_t)r * n_bins + b] = 2.0 * (double)counts[(size_t)r * n_bins + b] / (N * (N / V) * shell);
            }
        }
    }
    return check_device_errors(h);
}

// the records (cell order) and, when img is asked for, the image counts (site
// order), into the handle's host staging
static int fetch_records(mc_handle *h, const int4 **rec, const int **img)
{
    const size_t n = (size_t)h->n_sites;
    unsigned char *buf = (unsigned char *)h->host_buf(sizeof(int4) * n + (img ? sizeof(int) * 3 * n : 0));
    CUDA_TRY(cudaMemcpyAsync(buf, h->ds.rec[h->cur], sizeof(int4) * n, cudaMemcpyDeviceToHost, h->stream));
    if (img)
        CUDA_TRY(cudaMemcpyAsync(buf + sizeof(int4) * n, h->ds.img, sizeof(int) * 3 * n, cudaMemcpyDeviceToHost,
                                 h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    *rec = (const int4 *)buf;
    if (img) *img = (const int *)(buf + sizeof(int4) * n);
    return check_device_errors(h);
}

static int site_of(const mc_handle *h, int r, const int4 &v)
{
    return h->reps[r].site_off + 3 * (int)((uint32_t)v.w >> 4) + ((v.w >> 2) & 3);
}

int mc_state(mc_handle *h, double *xyz_out, int32_t *types_out, mc_stats *stats_out)
{
    if (!h) return fail(MC_ERR_INVALID_ARG, "NULL handle");
    int rc = set_device(h);
    if (rc) return rc;
    if (xyz_out || types_out) {
        const int4 *rec = nullptr;
        if ((rc = fetch_records(h, &rec, nullptr))) return rc;
        // on host threads, each taking a run of record slots (a replica's
        // records fill the slots of its sites; each record writes its own site)
        host_parallel((size_t)h->n_sites, 65536, [&](size_t b, size_t e) {
            int r = (int)(std::upper_bound(h->reps.begin(), h->reps.end(), b,
                                           [](size_t g, const RepInfo &ri) { return g < (size_t)ri.site_off; }) -
                          h->reps.begin()) - 1;
            for (size_t g = b; g < e; ++g) {
                while ((size_t)(h->reps[r].site_off + h->reps[r].n_sites) <= g) ++r;
                const RepInfo &ri = h->reps[r];
                const int4 v = rec[g];
                const int s = site_of(h, r, v);
                if (xyz_out) {
                    xyz_out[3 * (size_t)s + 0] = (double)(uint32_t)v.x * ri.h;
                    xyz_out[3 * (size_t)s + 1] = (double)(uint32_t)v.y * ri.h;
                    xyz_out[3 * (size_t)s + 2] = (double)(uint32_t)v.z * ri.h;
                }
                if (types_out) types_out[s] = v.w & 3;
            }
        });
    }
    if (stats_out) {
        std::vector<unsigned long long> st((size_t)STAT_N * h->n_rep);
        std::vector<double> e(h->n_rep), dr(2 * (size_t)h->n_rep);
        CUDA_TRY(cudaMemcpyAsync(st.data(), h->ds.stats, sizeof(unsigned long long) * st.size(), cudaMemcpyDeviceToHost,
                                 h->stream));
        CUDA_TRY(cudaMemcpyAsync(e.data(), h->ds.e_run, sizeof(double) * h->n_rep, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaMemcpyAsync(dr.data(), h->d_drift, sizeof(double) * dr.size(), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        for (int r = 0; r < h->n_rep; ++r) {
            mc_stats &s = stats_out[r];
            const unsigned long long *v = st.data() + (size_t)STAT_N * r;
            for (int k = 0; k < 4; ++k) {
                s.attempts[k] = v[STAT_ATT + k];
                s.accepts[k] = v[STAT_ACC + k];
            }
            s.rejected_geometry = v[STAT_REJ_GEOM];
            s.rejected_bond = v[STAT_REJ_BOND];
            s.pair_evals = v[STAT_PAIRS];
            s.fp64_rechecks = v[STAT_RECHECK];
            s.pair_interactions = v[STAT_INTER];
            s.sweeps = v[STAT_SWEEPS];
            s.e_run = e[r];
            s.recomputes = v[STAT_RECOMP];
            s.drift_last = dr[2 * (size_t)r];
            s.drift_max = dr[2 * (size_t)r + 1];
        }
        return check_device_errors(h);
    }
    return MC_OK;
}

int mc_state_fixed(mc_handle *h, uint32_t *q_out, int64_t *X_out, int32_t *types_out)
{
    if (!h) return fail(MC_ERR_INVALID_ARG, "NULL handle");
    int rc = set_device(h);
    if (rc) return rc;
    const int4 *rec = nullptr;
    const int *img = nullptr;
    if ((rc = fetch_records(h, &rec, &img))) return rc;
    for (int r = 0; r < h->n_rep; ++r) {
        const RepInfo &ri = h->reps[r];
        for (int i = 0; i < ri.n_sites; ++i) {
            const int4 v = rec[ri.site_off + i];
            const int s = site_of(h, r, v);
            const uint32_t q3[3] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z};
            for (int ax = 0; ax < 3; ++ax) {
                if (q_out) q_out[3 * (size_t)s + ax] = q3[ax];
                if (X_out) X_out[3 * (size_t)s + ax] = (int64_t)q3[ax] + ((int64_t)img[3 * (size_t)s + ax] << 32);
            }
            if (types_out) types_out[s] = v.w & 3;
        }
    }
    return MC_OK;
}

int mc_set_state(mc_handle *h, const double *xyz, const int32_t *types)
{
    if (!h || !xyz || !types) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    int rc = set_device(h);
    if (rc) return rc;
    int4 *rec = (int4 *)h->host_buf(sizeof(int4) * (size_t)h->n_sites);
    if ((rc = pack_records(h, xyz, nullptr, types, rec))) return rc;
    return rebuild_and_reset(h, rec);
}

int mc_set_state_fixed(mc_handle *h, const uint32_t *q, const int64_t *X, const int32_t *types)
{
    if (!h || !q || !types) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    int rc = set_device(h);
    if (rc) return rc;
    int4 *rec = (int4 *)h->host_buf(sizeof(int4) * (size_t)h->n_sites);
    if ((rc = pack_records(h, nullptr, q, types, rec))) return rc;
    if (!X) return rebuild_and_reset(h, rec);
    std::vector<int> img(3 * (size_t)h->n_sites);
    for (size_t k = 0; k < img.size(); ++k) {
        const int64_t d = X[k] - (int64_t)q[k];
        if (d % 4294967296LL != 0) return fail(MC_ERR_INVALID_ARG, "X - q is not a multiple of 2^32");
        img[k] = (int)(d / 4294967296LL);
    }
    return rebuild_and_reset(h, rec, &img);
}

int mc_set_sweep(mc_handle *h, uint64_t sweep)
{
    if (!h) return fail(MC_ERR_INVALID_ARG, "NULL handle");
    int rc = set_device(h);
    if (rc) return rc;
    std::vector<RepCtr> c(h->n_rep);
    CUDA_TRY(cudaMemcpyAsync(c.data(), h->d_ctr, sizeof(RepCtr) * h->n_rep, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (auto &x : c) x.sweep = sweep;
    CUDA_TRY(cudaMemcpyAsync(h->d_ctr, c.data(), sizeof(RepCtr) * h->n_rep, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return MC_OK;
}

int mc_reset_stats(mc_handle *h)
{
    if (!h) return fail(MC_ERR_INVALID_ARG, "NULL handle");
    int rc = set_device(h);
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(h->ds.stats, 0, sizeof(unsigned long long) * STAT_N * h->n_rep, h->stream));
    CUDA_TRY(cudaMemsetAsync(h->d_drift, 0, sizeof(double) * 2 * h->n_rep, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return MC_OK;
}

int mc_set_t0(mc_handle *h)
{
    if (!h) return fail(MC_ERR_INVALID_ARG, "NULL handle");
    int rc = set_device(h);
    if (rc) return rc;
    launch_gather(h->ds, h->cur, h->d_X, h->d_types, h->stream);
    launch_set_t0(h->ds, h->d_X, h->d_types, h->obs, h->stream);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->has_t0 = true;
    return MC_OK;
}

int mc_observables(mc_handle *h, const double *qvec_atom, int n_qa, const double *qvec_cm, int n_qc, double *out,
                   double *fs_atom, double *fscm_mol, double *c2_mol)
{
    if (!h || !qvec_atom || !qvec_cm || !out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    if (!h->has_t0) return fail(MC_ERR_INVALID_ARG, "mc_set_t0 has not been called");
    if (n_qa < 1 || n_qa > 256 || n_qc < 1 || n_qc > 256) return fail(MC_ERR_INVALID_ARG, "1 <= n_q <= 256");
    int rc = set_device(h);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(h->d_q, qvec_atom, sizeof(double) * 3 * n_qa, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->d_q + 3 * 256, qvec_cm, sizeof(double) * 3 * n_qc, cudaMemcpyHostToDevice, h->stream));
    launch_gather(h->ds, h->cur, h->d_X, h->d_types, h->stream);
    launch_observables(h->ds, h->d_X, h->obs, h->d_q, n_qa, h->d_q + 3 * 256, n_qc, h->d_fs, h->d_fscm, h->d_c2,
                       h->d_obs_out, h->stream);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(out, h->d_obs_out, sizeof(double) * 3 * h->n_rep, cudaMemcpyDeviceToHost, h->stream));
    const size_t M = (size_t)h->n_sites / 3;
    if (fs_atom)
        CUDA_TRY(cudaMemcpyAsync(fs_atom, h->d_fs, sizeof(double) * h->n_sites, cudaMemcpyDeviceToHost, h->stream));
    if (fscm_mol) CUDA_TRY(cudaMemcpyAsync(fscm_mol, h->d_fscm, sizeof(double) * M, cudaMemcpyDeviceToHost, h->stream));
    if (c2_mol) CUDA_TRY(cudaMemcpyAsync(c2_mol, h->d_c2, sizeof(double) * M, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return MC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Multiple-origin correlations
// ---------------------------------------------------------------------------
namespace {

template <class T>
int corr_alloc(mc_handle *h, T **p, size_t n)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return fail(MC_ERR_CUDA, std::string("cudaMalloc (correlation origins): ") + cudaGetErrorString(e));
    h->corr.bufs.push_back(q);
    *p = (T *)q;
    return MC_OK;
}

ObsState corr_slot(const mc_handle *h, int s)
{
    const size_t N = (size_t)h->n_sites, M = N / 3;
    ObsState o;
    o.X0 = const_cast<long long *>(h->corr.dev.X0) + (size_t)s * 3 * N;
    o.kref = const_cast<int *>(h->corr.dev.kref) + (size_t)s * M;
    o.u0 = const_cast<double *>(h->corr.dev.u0) + (size_t)s * 3 * M;
    return o;
}

// The decisions of the events at time t (host bookkeeping only): the live
// origins whose lag has come (slot, lag index), in slot order; then origins
// with t - t_o >= the last lag retire; then, at a multiple of every, the first
// free slot takes a new origin (new_slot, or -1).
struct CorrDecision {
    std::vector<std::pair<int, int>> pairs;
    int new_slot = -1;
};

CorrDecision corr_decide(std::vector<long long> &slot_t0, const std::vector<long long> &lags, int every, long long t)
{
    CorrDecision dd;
    const int n_slots = (int)slot_t0.size();
    for (int s = 0; s < n_slots; ++s) {
        if (slot_t0[s] < 0) continue;
        const auto it = std::lower_bound(lags.begin(), lags.end(), t - slot_t0[s]);
        if (it != lags.end() && *it == t - slot_t0[s]) dd.pairs.emplace_back(s, (int)(it - lags.begin()));
    }
    for (int s = 0; s < n_slots; ++s)
        if (slot_t0[s] >= 0 && t - slot_t0[s] >= lags.back()) slot_t0[s] = -1;
    if (t % every == 0) {
        int s = 0;
        while (s < n_slots && slot_t0[s] >= 0) ++s;
        if (s < n_slots) {
            slot_t0[s] = t;
            dd.new_slot = s;
        }
    }
    return dd;
}

// The events of the current time t: the samples (launched before any slot is
// reused), then the new origin and its lag-0 sample.
int corr_events(mc_handle *h)
{
    auto &c = h->corr;
    const CorrDecision dd = corr_decide(c.slot_t0, c.lags, c.every, c.t);
    bool gathered = false;
    CorrPairs p{};
    auto gather = [&]() {
        if (!gathered) launch_gather(h->ds, h->cur, h->d_X, h->d_types, h->stream);
        gathered = true;
    };
    auto flush = [&]() {
        if (p.n > 0) {
            gather();
            launch_corr_sample(h->ds, h->d_X, c.dev, p, h->stream);
        }
        p.n = 0;
    };
    for (const auto &sl : dd.pairs) {
        p.slot[p.n] = sl.first;
        p.lag[p.n] = sl.second;
        if (++p.n == kCorrMaxPairs) flush();
    }
    flush();
    if (dd.new_slot >= 0) {
        gather();
        launch_set_t0(h->ds, h->d_X, h->d_types, corr_slot(h, dd.new_slot), h->stream);
        if (c.lags[0] == 0) {
            p.slot[0] = dd.new_slot;
            p.lag[0] = 0;
            p.n = 1;
            flush();
        }
    }
    CUDA_TRY(cudaGetLastError());
    return MC_OK;
}

// The next time after t with an event: a multiple of origin_every, or a live
// origin's next lag.
long long corr_next(const mc_handle::Corr &c)
{
    long long nxt = (c.t / c.every + 1) * c.every;
    for (const long long t0 : c.slot_t0) {
        if (t0 < 0) continue;
        const auto it = std::upper_bound(c.lags.begin(), c.lags.end(), c.t - t0);
        if (it != c.lags.end()) nxt = std::min(nxt, t0 + *it);
    }
    return nxt;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

int corr_validate(int n_lags, const int64_t *lags, int origin_every, int max_origins)
{
    if (!lags) return fail(MC_ERR_INVALID_ARG, "NULL lags");
    if (n_lags < 1 || n_lags > 1024) return fail(MC_ERR_INVALID_ARG, "1 <= n_lags <= 1024");
    for (int l = 0; l < n_lags; ++l)
        if (lags[l] < 0 || (l > 0 && lags[l] <= lags[l - 1]))
            return fail(MC_ERR_INVALID_ARG, "lags must be strictly increasing and >= 0");
    if (origin_every < 1) return fail(MC_ERR_INVALID_ARG, "origin_every >= 1");
    if (max_origins < 1 || max_origins > 1024) return fail(MC_ERR_INVALID_ARG, "1 <= max_origins <= 1024");
    return MC_OK;
}

}  // namespace

extern "C" {

int mc_corr_schedule(int n_lags, const int64_t *lags, int origin_every, int max_origins, int64_t n_sweeps,
                     int64_t *counts)
{
    int rc = corr_validate(n_lags, lags, origin_every, max_origins);
    if (rc) return rc;
    if (!counts || n_sweeps < 0) return fail(MC_ERR_INVALID_ARG, "NULL counts or n_sweeps < 0");
    mc_handle::Corr c;
    c.lags.assign(lags, lags + n_lags);
    c.every = origin_every;
    c.slot_t0.assign(max_origins, -1);
    for (int l = 0; l < n_lags; ++l) counts[l] = 0;
    auto tally = [&]() {
        const CorrDecision dd = corr_decide(c.slot_t0, c.lags, c.every, c.t);
        for (const auto &sl : dd.pairs) counts[sl.second] += 1;
        if (dd.new_slot >= 0 && c.lags[0] == 0) counts[0] += 1;
    };
    c.t = 0;
    tally();
    while (true) {
        const long long nxt = corr_next(c);
        if (nxt > n_sweeps) break;
        c.t = nxt;
        tally();
    }
    return MC_OK;
}

int mc_corr_setup(mc_handle *h, int n_lags, const int64_t *lags, int origin_every, int max_origins,
                  const double *qvec_atom, int n_qa, const double *qvec_cm, int n_qc)
{
    if (!h || !lags || !qvec_atom || !qvec_cm) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    int rc = corr_validate(n_lags, lags, origin_every, max_origins);
    if (rc) return rc;
    if (n_qa < 1 || n_qa > 256 || n_qc < 1 || n_qc > 256) return fail(MC_ERR_INVALID_ARG, "1 <= n_q <= 256");
    rc = set_device(h);
    if (rc) return rc;
    corr_free(h);
    auto &c = h->corr;
    const size_t N = (size_t)h->n_sites, M = N / 3;
    // chunks of at most kCorrChunk molecules, none spanning two replicas
    std::vector<int> chunk_m0, rep_chunk0;
    for (int r = 0; r < h->n_rep; ++r) {
        rep_chunk0.push_back((int)chunk_m0.size());
        const int m_off = h->reps[r].site_off / 3, m_n = h->reps[r].n_sites / 3;
        for (int m = 0; m < m_n; m += kCorrChunk) chunk_m0.push_back(m_off + m);
    }
    const int n_chunks = (int)chunk_m0.size();
    rep_chunk0.push_back(n_chunks);
    chunk_m0.push_back((int)M);
    long long *X0 = nullptr;
    int *kref = nullptr, *cm0 = nullptr, *rc0 = nullptr;
    double *u0 = nullptr, *q = nullptr, *part = nullptr, *acc = nullptr;
    const size_t n_acc = (size_t)h->n_rep * n_lags * MC_CORR_NSUM;
    if ((rc = corr_alloc(h, &X0, (size_t)max_origins * 3 * N)) || (rc = corr_alloc(h, &kref, (size_t)max_origins * M)) ||
        (rc = corr_alloc(h, &u0, (size_t)max_origins * 3 * M)) || (rc = corr_alloc(h, &q, 3 * (size_t)(n_qa + n_qc))) ||
        (rc = corr_alloc(h, &cm0, chunk_m0.size())) || (rc = corr_alloc(h, &rc0, rep_chunk0.size())) ||
        (rc = corr_alloc(h, &part, (size_t)kCorrMaxPairs * n_chunks * kCorrPart)) || (rc = corr_alloc(h, &acc, n_acc))) {
        corr_free(h);
        return rc;
    }
    CUDA_TRY(cudaMemcpy(q, qvec_atom, sizeof(double) * 3 * n_qa, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(q + 3 * n_qa, qvec_cm, sizeof(double) * 3 * n_qc, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(cm0, chunk_m0.data(), sizeof(int) * chunk_m0.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(rc0, rep_chunk0.data(), sizeof(int) * rep_chunk0.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(acc, 0, sizeof(double) * n_acc));
    c.dev.X0 = X0;
    c.dev.kref = kref;
    c.dev.u0 = u0;
    c.dev.n_sites = N;
    c.dev.qa = q;
    c.dev.qc = q + 3 * n_qa;
    c.dev.n_qa = n_qa;
    c.dev.n_qc = n_qc;
    c.dev.chunk_m0 = cm0;
    c.dev.n_chunks = n_chunks;
    c.dev.rep_chunk0 = rc0;
    c.dev.partials = part;
    c.dev.acc = acc;
    c.dev.n_lags = n_lags;
    c.lags.assign(lags, lags + n_lags);
    c.every = origin_every;
    c.t = 0;
    c.slot_t0.assign(max_origins, -1);
    c.on = true;
    return corr_events(h);
}

int mc_corr_run(mc_handle *h, int n_sweeps, const double *T, const mc_move_mix *mix, const uint64_t *seeds)
{
    if (!h) return fail(MC_ERR_INVALID_ARG, "NULL handle");
    if (!h->corr.on) return fail(MC_ERR_INVALID_ARG, "mc_corr_setup has not been called");
    if (n_sweeps < 0 || !T || !mix || !seeds) return fail(MC_ERR_INVALID_ARG, "bad arguments");
    int left = n_sweeps;
    while (left > 0) {
        const long long nxt = corr_next(h->corr);
        const int k = (int)std::min<long long>(left, nxt - h->corr.t);
        int rc = sweep_impl(h, k, T, mix, seeds, false);
        if (rc) return rc;
        h->corr.t += k;
        left -= k;
        if (h->corr.t == nxt && (rc = corr_events(h))) return rc;
    }
    return MC_OK;
}

int mc_corr_sums(mc_handle *h, double *sums)
{
    if (!h || !sums) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    if (!h->corr.on) return fail(MC_ERR_INVALID_ARG, "mc_corr_setup has not been called");
    int rc = set_device(h);
    if (rc) return rc;
    const size_t n = (size_t)h->n_rep * h->corr.lags.size() * MC_CORR_NSUM;
    CUDA_TRY(cudaMemcpyAsync(sums, h->corr.dev.acc, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return MC_OK;
}

int mc_corr_derive(int n_rows, const double *sums, const int32_t *n_atoms, double *out)
{
    if (n_rows < 0 || (n_rows > 0 && (!sums || !n_atoms || !out))) return fail(MC_ERR_INVALID_ARG, "bad arguments");
    const double nan = std::nan("");
    for (int k = 0; k < n_rows; ++k) {
        if (n_atoms[k] < 3 || n_atoms[k] % 3 != 0) return fail(MC_ERR_INVALID_ARG, "n_atoms: a positive multiple of 3");
        const double N = (double)n_atoms[k], M = N / 3.0;
        const double *a = sums + (size_t)k * MC_CORR_NSUM;
        double *o = out + (size_t)k * MC_CORR_NRES;
        const double n = a[0];
        o[0] = n;
        if (!(n > 0.0)) {
            for (int j = 1; j < MC_CORR_NRES; ++j) o[j] = nan;
            continue;
        }
        const double fs = a[1] / n, fcm = a[5] / n, c2 = a[9] / n;
        o[1] = fs;
        o[2] = fcm;
        o[3] = c2;
        o[4] = N * (a[2] / n - fs * fs);
        o[5] = M * (a[6] / n - fcm * fcm);
        o[6] = M * (a[10] / n - c2 * c2);
        const double fs_i = a[3] / (n * N), fcm_i = a[7] / (n * M), c2_i = a[11] / (n * M);
        o[7] = a[4] / (n * N) - fs_i * fs_i;
        o[8] = a[8] / (n * M) - fcm_i * fcm_i;
        o[9] = a[12] / (n * M) - c2_i * c2_i;
        const double den = o[9] * o[8];
        o[10] = den > 0.0 ? (a[13] / (n * M) - c2_i * fcm_i) / std::sqrt(den) : nan;
    }
    return MC_OK;
}

int mc_corr_results(mc_handle *h, double *out)
{
    if (!h || !out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    if (!h->corr.on) return fail(MC_ERR_INVALID_ARG, "mc_corr_setup has not been called");
    const int nl = (int)h->corr.lags.size();
    std::vector<double> S((size_t)h->n_rep * nl * MC_CORR_NSUM);
    int rc = mc_corr_sums(h, S.data());
    if (rc) return rc;
    std::vector<int32_t> N((size_t)h->n_rep * nl);
    for (int r = 0; r < h->n_rep; ++r)
        for (int l = 0; l < nl; ++l) N[(size_t)r * nl + l] = h->reps[r].n_sites;
    return mc_corr_derive(h->n_rep * nl, S.data(), N.data(), out);
}

int mc_relaxation_time(int n_lags, const int64_t *lags, const double *values, const double *counts, double level,
                       double *tau)
{
    if (n_lags < 1 || !lags || !values || !counts || !tau) return fail(MC_ERR_INVALID_ARG, "bad arguments");
    *tau = std::nan("");
    double t_prev = 0.0, f_prev = 0.0;
    bool have_prev = false;
    for (int l = 0; l < n_lags; ++l) {
        if (!(counts[l] > 0.0)) continue;               // no sample at this lag
        const double t = (double)lags[l], f = values[l];
        if (f <= level) {
            if (!have_prev) {
                *tau = t;
            } else if (t_prev > 0.0) {
                // linear in ln t between the two lags that bracket the crossing
                const double a = (f_prev - level) / (f_prev - f);
                *tau = std::exp(std::log(t_prev) + a * (std::log(t) - std::log(t_prev)));
            } else {
                *tau = t_prev + (f_prev - level) / (f_prev - f) * (t - t_prev);
            }
            break;
        }
        t_prev = t;
        f_prev = f;
        have_prev = true;
    }
    return MC_OK;
}

int mc_corr_relaxation_time(mc_handle *h, int which, double level, double *tau)
{
    if (!h || !tau) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    if (which < 0 || which > 2) return fail(MC_ERR_INVALID_ARG, "which: 0 F_s, 1 F_s^cm, 2 C_2");
    if (!h->corr.on) return fail(MC_ERR_INVALID_ARG, "mc_corr_setup has not been called");
    const auto &lags = h->corr.lags;
    const int nl = (int)lags.size();
    std::vector<double> R((size_t)h->n_rep * nl * MC_CORR_NRES);
    int rc = mc_corr_results(h, R.data());
    if (rc) return rc;
    std::vector<int64_t> lg(lags.begin(), lags.end());
    std::vector<double> f(nl), n(nl);
    for (int r = 0; r < h->n_rep; ++r) {
        for (int l = 0; l < nl; ++l) {
            const double *o = R.data() + ((size_t)r * nl + l) * MC_CORR_NRES;
            n[l] = o[0];
            f[l] = o[1 + which];
        }
        if ((rc = mc_relaxation_time(nl, lg.data(), f.data(), n.data(), level, tau + r))) return rc;
    }
    return MC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Molecular dynamics
// ---------------------------------------------------------------------------
namespace {

// the cell-list build of an MD step draws no attempt random numbers
DevState md_state(const mc_handle *h)
{
    DevState d = h->ds;
    d.att_rnd = nullptr;
    return d;
}

// One MD step from the records of buf (the cell-sorted current buffer) into buf ^ 1, as a graph.
int md_graph(mc_handle *h, int buf)
{
    if (h->md.graph[buf]) return MC_OK;
    cudaStream_t cs;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const DevState d = md_state(h);
    launch_md_begin(d, h->md.dev, cs);
    launch_md_drift(d, buf, h->md.dev, cs);
    launch_cell_list(d, buf, buf ^ 1, cs);
    launch_md_forces(d, buf ^ 1, h->md.dev, cs);
    launch_md_end(d, h->md.dev, cs);
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(MC_ERR_CUDA, std::string("MD graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&h->md.graph[buf], g, 0);
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return fail(MC_ERR_CUDA, std::string("MD graph instantiate: ") + cudaGetErrorString(e));
    return MC_OK;
}

}  // namespace

extern "C" {

int mc_md_setup(mc_handle *h, double dt, double tau_T, const double *T, const double *v0, int force_precision)
{
    if (force_precision != MC_PREC_FP64 && force_precision != MC_PREC_FP32)
        return fail(MC_ERR_INVALID_ARG, "force_precision: MC_PREC_FP64 or MC_PREC_FP32");
    if (!h || !T || !v0) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(tau_T)) return fail(MC_ERR_INVALID_ARG, "dt > 0");
    for (int r = 0; r < h->n_rep; ++r)
        if (!(T[r] > 0.0) || !std::isfinite(T[r])) return fail(MC_ERR_INVALID_ARG, "temperature must be positive");
    int rc = set_device(h);
    if (rc) return rc;
    md_free(h);
    auto &m = h->md;
    const size_t N = (size_t)h->n_sites;
    m.T.assign(T, T + h->n_rep);
    m.Q.resize(h->n_rep);
    for (int r = 0; r < h->n_rep; ++r)   // tau_T <= 0: no thermostat (Q infinite, xi stays 0)
        m.Q[r] = tau_T > 0.0 ? 3.0 * h->reps[r].n_sites * T[r] * tau_T * tau_T : HUGE_VAL;
    // chunks of at most kMdChunk atoms, none spanning two replicas
    std::vector<int> chunk_a0, rep_chunk0;
    for (int r = 0; r < h->n_rep; ++r) {
        rep_chunk0.push_back((int)chunk_a0.size());
        for (int a = 0; a < h->reps[r].n_sites; a += kMdChunk) chunk_a0.push_back(h->reps[r].site_off + a);
    }
    const int n_chunks = (int)chunk_a0.size();
    rep_chunk0.push_back(n_chunks);
    chunk_a0.push_back((int)N);
    const size_t R = (size_t)h->n_rep;
    double *bufs[9] = {};
    const size_t sizes[9] = {3 * N, 3 * N, R, R, R, R, R, R, (size_t)n_chunks};
    int *ibufs[2] = {};
    const size_t isizes[2] = {chunk_a0.size(), rep_chunk0.size()};
    for (int k = 0; k < 11; ++k) {
        void *p = nullptr;
        const size_t bytes = k < 9 ? sizeof(double) * sizes[k] : sizeof(int) * isizes[k - 9];
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            md_free(h);
            return fail(MC_ERR_CUDA, std::string("cudaMalloc (MD): ") + cudaGetErrorString(e));
        }
        m.bufs.push_back(p);
        CUDA_TRY(cudaMemset(p, 0, bytes));
        if (k < 9) bufs[k] = (double *)p;
        else ibufs[k - 9] = (int *)p;
    }
    m.dev.v = bufs[0];
    m.dev.F = bufs[1];
    m.dev.xi = bufs[2];
    m.dev.eta = bufs[3];
    m.dev.K = bufs[4];
    m.dev.T = bufs[5];
    m.dev.Q = bufs[6];
    m.dev.scale = bufs[7];
    m.dev.part = bufs[8];
    m.dev.chunk_a0 = ibufs[0];
    m.dev.rep_chunk0 = ibufs[1];
    m.dev.n_chunks = n_chunks;
    m.dev.fp32_forces = force_precision == MC_PREC_FP32 ? 1 : 0;
    m.dev.dt = dt;
    m.dev.hdt = 0.5 * dt;
    CUDA_TRY(cudaMemcpy(ibufs[0], chunk_a0.data(), sizeof(int) * chunk_a0.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(ibufs[1], rep_chunk0.data(), sizeof(int) * rep_chunk0.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(bufs[0], v0, sizeof(double) * 3 * N, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(bufs[5], m.T.data(), sizeof(double) * h->n_rep, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(bufs[6], m.Q.data(), sizeof(double) * h->n_rep, cudaMemcpyHostToDevice));
    // the forces of the current state (its cell list is current)
    launch_md_forces(md_state(h), h->cur, m.dev, h->stream);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    m.on = true;
    return check_device_errors(h);
}

int mc_md_run(mc_handle *h, int n_steps)
{
    if (!h) return fail(MC_ERR_INVALID_ARG, "NULL handle");
    if (!h->md.on) return fail(MC_ERR_INVALID_ARG, "mc_md_setup has not been called");
    if (n_steps < 0) return fail(MC_ERR_INVALID_ARG, "n_steps < 0");
    int rc = set_device(h);
    if (rc) return rc;
    for (int s = 0; s < n_steps; ++s) {
        if ((rc = md_graph(h, h->cur))) return rc;
        CUDA_TRY(cudaGraphLaunch(h->md.graph[h->cur], h->stream));
        h->cur ^= 1;
    }
    // the running energy of later MC sweeps starts from the MD configuration
    if (n_steps > 0) {
        if ((rc = enqueue_energy(h))) return rc;
        CUDA_TRY(cudaMemcpyAsync(h->ds.e_run, h->d_e_out, sizeof(double) * h->n_rep, cudaMemcpyDeviceToDevice,
                                 h->stream));
    }
    CUDA_TRY(cudaGetLastError());
    return MC_OK;
}

int mc_md_state(mc_handle *h, double *v_out, double *out)
{
    if (!h || !out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    if (!h->md.on) return fail(MC_ERR_INVALID_ARG, "mc_md_setup has not been called");
    int rc = set_device(h);
    if (rc) return rc;
    const int R = h->n_rep;
    std::vector<double> v(3 * (size_t)h->n_sites), xi(R), eta(R), U(R);
    if ((rc = enqueue_energy(h))) return rc;
    CUDA_TRY(cudaMemcpyAsync(v.data(), h->md.dev.v, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(xi.data(), h->md.dev.xi, sizeof(double) * R, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(eta.data(), h->md.dev.eta, sizeof(double) * R, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(U.data(), h->d_e_out, sizeof(double) * R, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (v_out) std::memcpy(v_out, v.data(), sizeof(double) * v.size());
    for (int r = 0; r < R; ++r) {
        double K = 0.0;
        const size_t o = 3 * (size_t)h->reps[r].site_off, n = 3 * (size_t)h->reps[r].n_sites;
        for (size_t k = 0; k < n; ++k) K += 0.5 * v[o + k] * v[o + k];
        const double g = 3.0 * h->reps[r].n_sites;
        const double Q = h->md.Q[r];
        const double thermo = std::isfinite(Q) ? 0.5 * Q * xi[r] * xi[r] + g * h->md.T[r] * eta[r] : 0.0;
        out[5 * r + 0] = K;
        out[5 * r + 1] = U[r];
        out[5 * r + 2] = xi[r];
        out[5 * r + 3] = eta[r];
        out[5 * r + 4] = K + U[r] + thermo;
    }
    return check_device_errors(h);
}

int mc_get_info(mc_handle *h, mc_info *info)
{
    if (!h || !info) return fail(MC_ERR_INVALID_ARG, "NULL argument");
    info->n_rep = h->n_rep;
    info->precision = h->precision;
    info->stencil_cap = h->stencil_cap;
    info->total_sites = h->n_sites;
    info->total_cells = h->n_cells;
    int mx = 0;
    for (auto &r : h->reps) mx = std::max(mx, r.nc);
    info->max_cells_per_axis = mx;
    info->recheck_gap = h->recheck_gap;
    info->warps_per_cell = h->wpb;
    info->active_cells_per_colour = h->n_act;
    info->launch_mode = h->pgrid > 0 ? 2 : 1;
    info->persistent_blocks = h->pgrid;
    info->recompute_every = h->recompute_every;
    info->binary_version = sweep_binary_version();
    return MC_OK;
}

}  // extern "C"

extern "C" void mc_test_fail_alloc(int after)
{
    g_fail_alloc = after < 0 ? -1 : after;
}

int flipmc::record_error(int code, const char *msg)
{
    return fail(code, msg);
}

extern "C" {

const char *mc_last_error(void)
{
    return g_err.c_str();
}

}  // extern "C"
