// C ABI of librbe2d (declared in include/rbe2d.h): context management, argument
// checks and the launch sequence of one k-space force evaluation.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <string>
#include <vector>

#include "rbe2d_internal.h"
#include "rbe2d_setup.h"

using namespace rbe2d;

namespace rbe2d {
static std::atomic<unsigned long long> g_kernel_launches{0};
void note_launches(int n) { g_kernel_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
}  // namespace rbe2d

struct rbe2d_ctx {
    rbe2d_params p;
    DevParams dp;
    Shapes sh;
    int64_t n_max;
    cudaStream_t st;
    int device;
    bool fp64;
    // sampler tables
    double* cdf[3];
    int* guide[3];
    int cdf_len[3];
    double* wtab[3];      // the 1-D factors (Metropolis acceptance)
    double* eo_tab;       // image-series sums per kz of the sampler's box (9 float64 per row)
    SamplerTables tables;
    // Metropolis chains (one per batch slot)
    int32_t* mh_state;
    unsigned long long* mh_acc;
    bool mh_ready;
    // batch
    KCoef* kc;
    bool have_batch;
    // particles and partial sums
    void* part;
    double* pack_part;
    double* pack2;        // the pack rows summed in groups of 32 by the fold
    double* sf_part;
    int sf_nblk_max;
    double* rs;
    double* kterm;
    void* krec;
    double* scal;
    int* status;
    unsigned* counters;   // [0] fold CTAs done, [1] force rounds handed out, [2] force CTAs done,
                          // [3] real-space CTAs done, [4] MD kick CTAs done
    double* md_kpart;     // per-CTA kinetic-energy partial sums of the MD kick
    // real space
    bool real;
    CellGrid grid;
    RealBuffers rb;
    // pair lists of the MD loop
    bool lists = false;
    PairLists nl = {};
    int64_t nl_N = -1;  // N of the last list evaluation (another N forces a rebuild)
    // staging for RBE2D_HOST_BUFFERS
    double* stage_in;     // n_max * 3 (pos) + n_max (q)
    void* stage_out;      // n_max * 3 outputs (force or dpos)
    void* stage_out2;     // n_max outputs (phi or dq)
    double* stage_small;  // 8 doubles
    // FMA-pipe sin/cos share and launch shape of the FP32 kernels (set by rbe2d_autotune;
    // the defaults are the tuner's choice at N = 1e6, P = 500 on GB300)
    int sf_poly = 2, f_poly = 1;
    int sf_shape = 0, f_shape = 4;
    // the same for the force kernel's potential variant (rbe2d_autotune_potential)
    int p_poly = 0, p_shape = 0;
    // state of the last structure-factor evaluation
    bool sf_valid;
    int64_t sf_N;
    int sf_sigma;
    bool ureal_set = false;  // scal[SC_UREAL] holds a real-space energy (the fold clears it)
    // per-kernel timer: 2 * tcap events per class (start, end), tn[cls] pairs recorded
    int tcap = 0;
    unsigned tmask = 0;
    std::vector<cudaEvent_t> tev[RBE2D_TIMER_COUNT];
    int tn[RBE2D_TIMER_COUNT] = {};
    std::string err;
};

namespace {

thread_local std::string g_init_error;  // message of the last failed rbe2d_init on this thread

int fail(rbe2d_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_fail(rbe2d_ctx* c, cudaError_t e, const char* where) {
    return fail(c, RBE2D_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                     \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

void timer_free(rbe2d_ctx* c) {
    for (int k = 0; k < RBE2D_TIMER_COUNT; k++) {
        for (cudaEvent_t e : c->tev[k]) cudaEventDestroy(e);
        c->tev[k].clear();
        c->tn[k] = 0;
    }
    c->tcap = 0;
    c->tmask = 0;
}

// Records a start event on construction and an end event on destruction around the
// launches of one kernel class, when the timer is on, has room and the stream is not
// being captured.
struct KTimer {
    rbe2d_ctx* c;
    int cls;
    bool on = false;
    KTimer(rbe2d_ctx* ctx, int k) : c(ctx), cls(k) {
        if (c->tcap == 0 || !(c->tmask >> k & 1u) || c->tn[k] >= c->tcap) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(c->st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
        on = cudaEventRecord(c->tev[k][2 * c->tn[k]], c->st) == cudaSuccess;
    }
    ~KTimer() {
        if (on && cudaEventRecord(c->tev[cls][2 * c->tn[cls] + 1], c->st) == cudaSuccess) c->tn[cls]++;
    }
};

size_t part_bytes(bool fp64) { return fp64 ? sizeof(Part64) : sizeof(uint4); }

// The tuned FMA-pipe share and shape of a force launch: the potential variant's choice
// when the launch writes dU/dq (phi set), the plain force's otherwise.
int force_poly(const rbe2d_ctx* c, const void* phi) { return phi ? c->p_poly : c->f_poly; }
int force_shape(const rbe2d_ctx* c, const void* phi) { return phi ? c->p_shape : c->f_shape; }

void free_all(rbe2d_ctx* c) {
    timer_free(c);
    for (int d = 0; d < 3; d++) {
        cudaFree(c->cdf[d]);
        cudaFree(c->guide[d]);
        cudaFree(c->wtab[d]);
    }
    cudaFree(c->eo_tab);
    cudaFree(c->kc);
    cudaFree(c->mh_state);
    cudaFree(c->mh_acc);
    cudaFree(c->part);
    cudaFree(c->pack_part);
    cudaFree(c->pack2);
    cudaFree(c->sf_part);
    cudaFree(c->rs);
    cudaFree(c->kterm);
    cudaFree(c->krec);
    cudaFree(c->scal);
    cudaFree(c->status);
    cudaFree(c->counters);
    cudaFree(c->md_kpart);
    cudaFree(c->rb.count);
    cudaFree(c->rb.start);
    cudaFree(c->rb.fill);
    cudaFree(c->rb.tile_sum);
    cudaFree(c->rb.src);
    cudaFree(c->rb.src_sorted);
    cudaFree(c->rb.key);
    cudaFree(c->rb.key_sorted);
    cudaFree(c->rb.epart);
    cudaFree(c->nl.nl);
    cudaFree(c->nl.cnt);
    cudaFree(c->nl.tgt);
    cudaFree(c->nl.rec);
    cudaFree(c->nl.ref);
    cudaFree(c->nl.srec);
    cudaFree(c->nl.inv);
    cudaFree(c->nl.count_real);
    cudaFree(c->nl.real_start);
    cudaFree(c->nl.tile_sum2);
    cudaFree(c->nl.flag);
    cudaFree(c->nl.builds);
    cudaFree(c->stage_in);
    cudaFree(c->stage_out);
    cudaFree(c->stage_out2);
    cudaFree(c->stage_small);
}

// Real-space cell grid for cutoff rcut: cells of at least rcut in x, y (periodic) and in z
// over [-rcut, H + rcut] (at most 16e6 cells), images up to the level that can reach
// within rcut of the slab.
CellGrid make_grid(const rbe2d_params& p, double rcut, bool diel) {
    CellGrid g;
    g.ncx = (int)floor(p.Lx / rcut); if (g.ncx < 1) g.ncx = 1;
    g.ncy = (int)floor(p.Ly / rcut); if (g.ncy < 1) g.ncy = 1;
    g.ncz = (int)floor((p.H + 2.0 * rcut) / rcut); if (g.ncz < 1) g.ncz = 1;
    if ((double)g.ncx * g.ncy * g.ncz > 16.0e6) {
        const double f = cbrt((double)g.ncx * g.ncy * g.ncz / 16.0e6);
        g.ncx = (int)(g.ncx / f) > 0 ? (int)(g.ncx / f) : 1;
        g.ncy = (int)(g.ncy / f) > 0 ? (int)(g.ncy / f) : 1;
        g.ncz = (int)(g.ncz / f) > 0 ? (int)(g.ncz / f) : 1;
    }
    g.ncell = g.ncx * g.ncy * g.ncz;
    g.hx = p.Lx / g.ncx; g.hy = p.Ly / g.ncy; g.hz = (p.H + 2.0 * rcut) / g.ncz; g.z0 = -rcut;
    g.inv_hx = 1.0 / g.hx; g.inv_hy = 1.0 / g.hy; g.inv_hz = 1.0 / g.hz;
    g.mx = (int)ceil(rcut / g.hx); g.my = (int)ceil(rcut / g.hy);
    const int lreach = 2 + (int)ceil(rcut / p.H);
    g.lmax = diel ? (p.M < lreach ? p.M : lreach) : 0;
    return g;
}

// pack -> structure factor -> fold -> finalize, on device inputs (or on pinned host
// inputs read in place: host_inputs).
int run_sf(rbe2d_ctx* c, int64_t N, const void* pos, const void* q, bool in_f32, bool want_sigma,
           bool host_inputs = false) {
    const DevParams& dp = c->dp;
    // the tuned shape applies to float64 inputs in device memory; other inputs run shape 0
    const int shape = (c->fp64 || in_f32 || host_inputs) ? 0 : c->sf_shape;
    int threads = c->fp64 ? c->sh.sf_threads64 : c->sh.sf_threads32[shape];
    int kr = c->fp64 ? 2 : kSfKR[shape];
    int occ = c->fp64 ? c->sh.sf_occ64 : c->sh.sf_occ32[shape];
    int kchunks = (dp.P + threads * kr - 1) / (threads * kr);
    // at least 64 particles per CTA: a small system still spreads over the SMs (the cap
    // below keeps a large one at one wave)
    int64_t want = (N + 63) / 64;
    int nblk = (int)(want < 1 ? 1 : want);
    // one wave of resident CTAs over the k chunks, within the partial-sum buffer
    int cap = c->sh.sms * occ / kchunks;
    if (cap > c->sf_nblk_max / kchunks) cap = c->sf_nblk_max / kchunks;
    if (cap < 1) cap = 1;
    if (nblk > cap) nblk = cap;
    int pb;
    if (c->fp64) {
        pb = pack_blocks_for(N);
        {
            KTimer kt(c, RBE2D_TIMER_PACK);
            CK(launch_pack(c->st, dp, N, pos, q, in_f32, true, c->part, c->pack_part, pb), "pack launch");
        }
        KTimer kt(c, RBE2D_TIMER_SF);
        CK(launch_sf64(c->st, dp, N, c->part, want_sigma, c->kc, c->sf_part, nblk, threads, kchunks),
           "structure factor launch");
    } else {
        pb = nblk;  // the structure-factor CTAs of the first k-chunk write the pack sums
        KTimer kt(c, RBE2D_TIMER_SF);
        CK(launch_sf32(c->st, dp, N, pos, q, in_f32, want_sigma, c->kc, c->sf_part, nblk, threads, kchunks, c->part,
                       c->pack_part, c->sf_poly, host_inputs, shape),
           "structure factor launch");
    }
    {
        KTimer kt(c, RBE2D_TIMER_FOLD);
        CK(launch_fold(c->st, dp, c->sf_part, nblk, c->kc, c->fp64, c->rs, c->kterm, c->krec, c->pack_part, pb,
                       c->pack2, c->scal, c->counters),
           "fold launch");
    }
    c->sf_valid = true;
    c->ureal_set = false;
    c->sf_N = N;
    c->sf_sigma = want_sigma ? 1 : 0;
    return RBE2D_OK;
}

// Device address of host memory the GPU can reach directly (pinned or registered host
// memory, mapped under unified addressing; on Grace hosts the accesses go over
// NVLink-C2C), or NULL.
void* device_view(const void* h) {
    if (!h) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

int check_common(rbe2d_ctx* c, int64_t N, const void* pos, const void* q) {
    if (!c) return RBE2D_EINVAL;
    if (N < 0 || N > c->n_max) return fail(c, RBE2D_EINVAL, "N = %lld outside [0, n_max = %lld]", (long long)N, (long long)c->n_max);
    if (N > 0 && (!pos || !q)) return fail(c, RBE2D_EINVAL, "pos and q must not be NULL");
    if (!c->have_batch) return fail(c, RBE2D_EINVAL, "no k batch: call rbe2d_sample_k or rbe2d_set_k first");
    return RBE2D_OK;
}

// Copy host inputs into the staging buffer; returns device pointers.
int stage_inputs(rbe2d_ctx* c, int64_t N, const void* pos, const void* q, bool in_f32, const void** dpos,
                 const void** dq) {
    size_t es = in_f32 ? sizeof(float) : sizeof(double);
    char* base = reinterpret_cast<char*>(c->stage_in);
    CK(cudaMemcpyAsync(base, pos, (size_t)N * 3 * es, cudaMemcpyHostToDevice, c->st), "copy pos to device");
    char* qd = base + (size_t)c->n_max * 3 * sizeof(double);
    CK(cudaMemcpyAsync(qd, q, (size_t)N * es, cudaMemcpyHostToDevice, c->st), "copy q to device");
    *dpos = base;
    *dq = qd;
    return RBE2D_OK;
}

int validate(rbe2d_ctx* c) {
    double s[SC_COUNT];
    CK(cudaMemcpyAsync(s, c->scal, sizeof s, cudaMemcpyDeviceToHost, c->st), "read validation sums");
    CK(cudaStreamSynchronize(c->st), "synchronise");
    if (fabs(s[SC_Q]) > 1e-10 * s[SC_QABS] + 1e-300)
        return fail(c, RBE2D_ENONNEUTRAL, "total charge %.17g is not zero (sum |q| = %.17g)", s[SC_Q], s[SC_QABS]);
    if (s[SC_ZMIN] < 0.0 || s[SC_ZMAX] > c->dp.H)
        return fail(c, RBE2D_ERANGE, "z range [%.17g, %.17g] leaves the slab [0, %.17g]", s[SC_ZMIN], s[SC_ZMAX], c->dp.H);
    return RBE2D_OK;
}

}  // namespace

extern "C" {

int rbe2d_init(const rbe2d_params* params, int64_t n_max, void* stream, rbe2d_ctx** out) {
    if (!params || !out) return RBE2D_EINVAL;
    *out = nullptr;
    rbe2d_ctx* c = new (std::nothrow) rbe2d_ctx();
    if (!c) return RBE2D_ENOMEM;
    rbe2d_params p = *params;
    auto bad = [&](const char* msg) {
        g_init_error = msg;
        delete c;
        return RBE2D_EINVAL;
    };
    g_init_error.clear();
    if (!(p.Lx > 0) || !(p.Ly > 0) || !(p.H > 0)) return bad("Lx, Ly, H must be positive");
    if (!(fabs(p.gamma_top) <= 1.0) || !(fabs(p.gamma_bot) <= 1.0)) return bad("|gamma| must be <= 1");
    if (p.P < 1 || p.P > 65536) return bad("P must be in [1, 65536]");
    if (n_max < 1) return bad("n_max must be >= 1");
    if (p.precision != RBE2D_FP64 && p.precision != RBE2D_FP32_MIXED) return bad("unknown precision");
    if (!(p.eps > 0)) p.eps = 1e-4;
    if (!(p.eps < 1)) return bad("eps must be < 1");
    if (!(p.coulomb_k > 0)) p.coulomb_k = 1.0;
    if (!(p.alpha > 0)) p.alpha = cbrt((double)n_max / (p.Lx * p.Ly * p.H));
    if (p.M < 0) p.M = auto_M(p.Lx, p.Ly, p.H, p.gamma_top, p.gamma_bot, p.eps);
    if (p.M > 1024) return bad("M must be <= 1024");
    if (!(p.Lz > 0)) p.Lz = auto_Lz(p.Lx, p.Ly, p.H, p.M, p.alpha, p.eps);
    if (p.Lz < (p.M + 1) * p.H) return bad("Lz < (M+1) H (Eq. 3.23)");
    if (!(p.r_c > 0)) p.r_c = 3.0 / p.alpha;
    c->p = p;
    c->n_max = n_max;
    c->st = (cudaStream_t)stream;
    c->fp64 = p.precision == RBE2D_FP64;
    cudaGetDevice(&c->device);

    // host tables and constants
    std::vector<double> cdf[3];
    const double Ls[3] = {p.Lx, p.Ly, p.Lz};
    double Sd[3];
    for (int d = 0; d < 3; d++) Sd[d] = build_cdf(p.alpha, Ls[d], &cdf[d]);
    ImageConsts ic;
    image_constants(p.gamma_top, p.gamma_bot, p.M, &ic);
    DevParams& dp = c->dp;
    dp.Lx = p.Lx; dp.Ly = p.Ly; dp.H = p.H; dp.Lz = p.Lz; dp.V = p.Lx * p.Ly * p.Lz;
    dp.inv_Lx = 1.0 / p.Lx; dp.inv_Ly = 1.0 / p.Ly; dp.inv_Lz = 1.0 / p.Lz;
    dp.S = Sd[0] * Sd[1] * Sd[2] - 1.0;
    dp.alpha = p.alpha; dp.r_c = p.r_c; dp.gt = p.gamma_top; dp.gb = p.gamma_bot; dp.kc = p.coulomb_k;
    dp.coef = 2.0 * M_PI / dp.V * (dp.S / p.P) * p.coulomb_k;
    dp.coef_unit = 2.0 * M_PI / dp.V * p.coulomb_k;
    dp.self_c = -p.alpha / sqrt(M_PI) * p.coulomb_k;
    dp.cM = ic.cM; dp.dM = ic.dM; dp.dcM_t = ic.dcM_t; dp.dcM_b = ic.dcM_b; dp.ddM_t = ic.ddM_t; dp.ddM_b = ic.ddM_b;
    dp.M = p.M; dp.P = p.P; dp.P_pad = ((p.P + 31) / 32) * 32;
    dp.diel = (p.M > 0 && (p.gamma_top != 0.0 || p.gamma_bot != 0.0)) ? 1 : 0;
    dp.kseg = 4;
    while (dp.kseg < 32 && dp.kseg < p.M / 2 + 1) dp.kseg *= 2;

    cudaError_t e = query_shapes(c->device, dp.P_pad, &c->sh);
    if (e != cudaSuccess) {
        g_init_error = std::string("query launch shapes: ") + cudaGetErrorString(e);
        delete c;
        return RBE2D_ECUDA;
    }
    // partial-sum rows for the largest one-wave grid of any structure-factor shape
    c->sf_nblk_max = 0;
    int kchunks = 1;
    for (int v = 0; v < (c->fp64 ? 1 : kSfShapes); v++) {
        const int threads = c->fp64 ? c->sh.sf_threads64 : c->sh.sf_threads32[v];
        const int occ = c->fp64 ? c->sh.sf_occ64 : c->sh.sf_occ32[v];
        const int kr = c->fp64 ? 2 : kSfKR[v];
        const int kc_v = (dp.P + threads * kr - 1) / (threads * kr);
        if (c->sh.sms * occ > c->sf_nblk_max) c->sf_nblk_max = c->sh.sms * occ;
        if (kc_v > kchunks) kchunks = kc_v;
    }
    // keep the per-chunk partial sums (P_pad x nblk x 4 doubles) under 256 MB
    const int64_t cap = (int64_t)(256u << 20) / (32 * (int64_t)dp.P_pad);
    if (c->sf_nblk_max > cap) c->sf_nblk_max = (int)cap;
    if (c->sf_nblk_max < kchunks) c->sf_nblk_max = kchunks;

    bool ok = true;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(ptr, bytes < 16 ? 16 : bytes) != cudaSuccess) ok = false;
    };
    std::vector<int> guide[3];
    std::vector<double> wt[3];
    for (int d = 0; d < 3; d++) {
        build_guide(cdf[d], &guide[d]);
        build_weights(p.alpha, Ls[d], &wt[d]);
        c->cdf_len[d] = (int)cdf[d].size();
        alloc((void**)&c->cdf[d], cdf[d].size() * sizeof(double));
        alloc((void**)&c->guide[d], guide[d].size() * sizeof(int));
        alloc((void**)&c->wtab[d], wt[d].size() * sizeof(double));
    }
    alloc((void**)&c->kc, sizeof(KCoef) * dp.P_pad);
    alloc((void**)&c->eo_tab, sizeof(double) * 9 * (size_t)(cdf[2].size()));
    alloc((void**)&c->mh_state, sizeof(int32_t) * 3 * (size_t)dp.P_pad);
    alloc((void**)&c->mh_acc, sizeof(unsigned long long));
    alloc(&c->part, part_bytes(c->fp64) * (size_t)n_max);
    alloc((void**)&c->pack_part, sizeof(double) * PACK_STRIDE * (size_t)(c->sf_nblk_max > 1024 ? c->sf_nblk_max : 1024));
    alloc((void**)&c->pack2, sizeof(double) * PACK_STRIDE * (size_t)((c->sf_nblk_max > 1024 ? c->sf_nblk_max : 1024) / 32 + 2));
    alloc((void**)&c->sf_part, sizeof(double) * 4 * (size_t)dp.P_pad * c->sf_nblk_max);
    alloc((void**)&c->rs, sizeof(double) * 4 * dp.P_pad);
    alloc((void**)&c->kterm, sizeof(double) * 3 * dp.P_pad);
    alloc(&c->krec, c->fp64 ? sizeof(KRec64) * dp.P_pad : sizeof(KPair32) * (dp.P_pad / 2));
    alloc((void**)&c->scal, sizeof(double) * SC_COUNT);
    alloc((void**)&c->status, sizeof(int) * ST_COUNT);
    alloc((void**)&c->counters, sizeof(unsigned) * 8);
    alloc((void**)&c->md_kpart, sizeof(double) * (size_t)md_blocks(n_max));
    alloc((void**)&c->stage_in, sizeof(double) * 4 * (size_t)n_max);
    alloc(&c->stage_out, sizeof(double) * 3 * (size_t)n_max);
    alloc(&c->stage_out2, sizeof(double) * (size_t)n_max);
    alloc((void**)&c->stage_small, sizeof(double) * 8);
    if (p.real_space) {
        // cells of at least r_c; images up to the level that can reach within r_c of the slab
        CellGrid& g = c->grid;
        g = make_grid(p, p.r_c, dp.diel != 0);
        int64_t ncell_max = g.ncell;
        int lmax = g.lmax;
        // pair lists of the MD loop: float32 mode, a box wide enough for the fixed-point
        // minimum image of pairs within r_c + 2 skin, list entries within 31 bits
        const double rcs = p.r_c + p.skin;
        c->lists = p.skin > 0 && !c->fp64 && p.Lx >= 2.0 * (p.r_c + 2.0 * p.skin) &&
                   p.Ly >= 2.0 * (p.r_c + 2.0 * p.skin) && n_max < (int64_t)1 << 25;
        if (c->lists) {
            PairLists& L = c->nl;
            L.skin = p.skin;
            L.g = make_grid(p, rcs, dp.diel != 0);
            if (2 * L.g.lmax + 1 > kNlMaxSlots) c->lists = false;
            if (L.g.ncell > ncell_max) ncell_max = L.g.ncell;
            if (L.g.lmax > lmax) lmax = L.g.lmax;
            // capacity: twice the mean number of sources within r_c + skin (the image layers
            // continue the slab's density), plus a margin for crowded charges
            const double rho = (double)n_max / (p.Lx * p.Ly * p.H);
            const double mean = rho * 4.0 / 3.0 * M_PI * rcs * rcs * rcs;
            int64_t cap = (int64_t)(2.0 * mean) + 64;
            cap = (cap + 31) / 32 * 32;
            if (cap > 4096) cap = 4096;
            L.cap = (int)cap;
            L.n_slots = n_max;
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1)
                sms = 1;
            L.build_blocks = 8 * sms;
            alloc((void**)&L.nl, sizeof(int) * (size_t)L.cap * (size_t)n_max);
            alloc((void**)&L.cnt, sizeof(int) * (size_t)n_max);
            alloc((void**)&L.tgt, sizeof(int) * (size_t)n_max);
            alloc((void**)&L.rec, sizeof(uint4) * (size_t)n_max);
            alloc((void**)&L.ref, sizeof(uint4) * (size_t)n_max);
            alloc((void**)&L.srec, sizeof(uint4) * (size_t)n_max);
            alloc((void**)&L.inv, sizeof(int) * (size_t)n_max);
            alloc((void**)&L.count_real, sizeof(int) * (size_t)L.g.ncell);
            alloc((void**)&L.real_start, sizeof(int) * ((size_t)L.g.ncell + 1));
            alloc((void**)&L.tile_sum2, sizeof(int) * (size_t)((L.g.ncell + 1023) / 1024));
            alloc((void**)&L.flag, sizeof(int) * 4);
            alloc((void**)&L.builds, sizeof(unsigned long long));
        }
        RealBuffers& rb = c->rb;
        rb.nsrc_max = n_max * (int64_t)(1 + 2 * lmax);
        const size_t vs = c->fp64 ? 32 : 16;
        alloc((void**)&rb.count, sizeof(int) * (size_t)ncell_max);
        alloc((void**)&rb.start, sizeof(int) * ((size_t)ncell_max + 1));
        alloc((void**)&rb.fill, sizeof(int) * (size_t)ncell_max);
        alloc((void**)&rb.tile_sum, sizeof(int) * (size_t)((ncell_max + 1023) / 1024));
        alloc(&rb.src, vs * (size_t)rb.nsrc_max);
        alloc(&rb.src_sorted, vs * (size_t)rb.nsrc_max);
        alloc((void**)&rb.key, sizeof(long long) * (size_t)rb.nsrc_max);
        alloc((void**)&rb.key_sorted, sizeof(long long) * (size_t)rb.nsrc_max);
        alloc((void**)&rb.epart, sizeof(double) * (size_t)ncell_max);
        c->real = true;
        if (rb.nsrc_max > 2000000000LL) ok = false;
    }
    if (!ok) {
        cudaGetLastError();
        g_init_error = "device allocation failed";
        free_all(c);
        delete c;
        return RBE2D_ENOMEM;
    }
    for (int d = 0; d < 3; d++) {
        e = cudaMemcpy(c->cdf[d], cdf[d].data(), cdf[d].size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->guide[d], guide[d].data(), guide[d].size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->wtab[d], wt[d].data(), wt[d].size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) break;
        c->tables.cdf[d] = c->cdf[d];
        c->tables.guide[d] = c->guide[d];
        c->tables.w[d] = c->wtab[d];
        c->tables.len[d] = c->cdf_len[d];
        c->tables.hw[d] = metropolis_half_width(p.alpha, Ls[d]);
    }
    if (e == cudaSuccess) {  // the image-series table of every kz the samplers can draw
        c->tables.eo = c->eo_tab;
        c->tables.eo_half = c->cdf_len[2] / 2;
        e = launch_eo_table(0, dp, c->tables.eo_half, c->eo_tab);
    }
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(int) * ST_COUNT);
    if (e == cudaSuccess) e = cudaMemset(c->counters, 0, sizeof(unsigned) * 8);
    if (e == cudaSuccess) e = cudaMemset(c->scal, 0, sizeof(double) * SC_COUNT);
    if (e == cudaSuccess && c->lists) e = cudaMemset(c->nl.flag, 1, sizeof(int) * 4);  // build before the first use
    if (e == cudaSuccess && c->lists) e = cudaMemset(c->nl.builds, 0, sizeof(unsigned long long));
    if (e == cudaSuccess && c->lists) e = cudaMemset(c->nl.inv, 0, sizeof(int) * (size_t)n_max);
    // FP32 records: the k1 half of the last pair stays zero when P is odd
    if (e == cudaSuccess && !c->fp64) e = cudaMemset(c->krec, 0, sizeof(KPair32) * (dp.P_pad / 2));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        g_init_error = std::string("device setup: ") + cudaGetErrorString(e);
        free_all(c);
        delete c;
        return RBE2D_ECUDA;
    }
    *out = c;
    return RBE2D_OK;
}

int rbe2d_destroy(rbe2d_ctx* c) {
    if (!c) return RBE2D_OK;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->st);
    free_all(c);
    delete c;
    return RBE2D_OK;
}

const char* rbe2d_last_error(const rbe2d_ctx* c) { return c ? c->err.c_str() : g_init_error.c_str(); }

int rbe2d_get_derived(const rbe2d_ctx* c, double* S, double* Lz, int* M, double* alpha, double* r_c) {
    if (!c) return RBE2D_EINVAL;
    if (S) *S = c->dp.S;
    if (Lz) *Lz = c->dp.Lz;
    if (M) *M = c->dp.M;
    if (alpha) *alpha = c->dp.alpha;
    if (r_c) *r_c = c->dp.r_c;
    return RBE2D_OK;
}

int rbe2d_sample_k(rbe2d_ctx* c, uint64_t step, int32_t* k_idx_out) {
    if (!c) return RBE2D_EINVAL;
    DeviceGuard g(c->device);
    KTimer kt(c, RBE2D_TIMER_SAMPLE);
    CK(launch_sample(c->st, c->dp, c->tables, c->p.seed, step, nullptr, c->kc, k_idx_out, c->status),
       "sample launch");
    c->have_batch = true;
    c->sf_valid = false;
    return RBE2D_OK;
}

int rbe2d_sample_k_dev(rbe2d_ctx* c, const uint64_t* step_dev, int32_t* k_idx_out) {
    if (!c) return RBE2D_EINVAL;
    if (!step_dev) return fail(c, RBE2D_EINVAL, "step_dev must not be NULL");
    DeviceGuard g(c->device);
    KTimer kt(c, RBE2D_TIMER_SAMPLE);
    CK(launch_sample(c->st, c->dp, c->tables, c->p.seed, 0, (const unsigned long long*)step_dev, c->kc, k_idx_out,
                     c->status),
       "sample launch");
    c->have_batch = true;
    c->sf_valid = false;
    return RBE2D_OK;
}

int rbe2d_metropolis_reset(rbe2d_ctx* c, const int32_t* k_start) {
    if (!c) return RBE2D_EINVAL;
    DeviceGuard g(c->device);
    if (k_start) {
        CK(cudaMemcpyAsync(c->mh_state, k_start, sizeof(int32_t) * 3 * (size_t)c->dp.P, cudaMemcpyDeviceToDevice,
                           c->st),
           "copy chain starts");
    } else {  // stationary start: the i.i.d. draw of step 0
        CK(launch_sample(c->st, c->dp, c->tables, c->p.seed, 0, nullptr, c->kc, c->mh_state, c->status),
           "sample launch");
    }
    CK(cudaMemsetAsync(c->mh_acc, 0, sizeof(unsigned long long), c->st), "clear acceptance count");
    c->mh_ready = true;
    return RBE2D_OK;
}

int rbe2d_sample_k_metropolis(rbe2d_ctx* c, uint64_t step, int sweeps, int32_t* k_idx_out) {
    if (!c) return RBE2D_EINVAL;
    if (!c->mh_ready) return fail(c, RBE2D_EINVAL, "call rbe2d_metropolis_reset first");
    if (sweeps < 1 || sweeps > (1 << 20)) return fail(c, RBE2D_EINVAL, "sweeps = %d outside [1, 2^20]", sweeps);
    DeviceGuard g(c->device);
    KTimer kt(c, RBE2D_TIMER_SAMPLE);
    CK(launch_metropolis(c->st, c->dp, c->tables, c->p.seed, step, sweeps, c->mh_state, c->kc, k_idx_out, c->mh_acc),
       "Metropolis launch");
    c->have_batch = true;
    c->sf_valid = false;
    return RBE2D_OK;
}

int rbe2d_metropolis_accepted(rbe2d_ctx* c, uint64_t* accepted_out) {
    if (!c) return RBE2D_EINVAL;
    if (!accepted_out) return fail(c, RBE2D_EINVAL, "accepted_out must not be NULL");
    DeviceGuard g(c->device);
    unsigned long long a = 0;
    CK(cudaMemcpyAsync(&a, c->mh_acc, sizeof a, cudaMemcpyDeviceToHost, c->st), "read acceptance count");
    CK(cudaStreamSynchronize(c->st), "synchronise");
    *accepted_out = a;
    return RBE2D_OK;
}

int rbe2d_set_k(rbe2d_ctx* c, const int32_t* k_idx) {
    if (!c) return RBE2D_EINVAL;
    if (!k_idx) return fail(c, RBE2D_EINVAL, "k_idx must not be NULL");
    DeviceGuard g(c->device);
    CK(launch_set_k(c->st, c->dp, k_idx, c->kc, c->status), "set_k launch");
    c->have_batch = true;
    c->sf_valid = false;
    return RBE2D_OK;
}

int rbe2d_structure_factor(rbe2d_ctx* c, int64_t N, const void* pos, const void* q, int flags, double* rho_out) {
    int r = check_common(c, N, pos, q);
    if (r) return r;
    DeviceGuard g(c->device);
    const bool in_f32 = (flags & RBE2D_INPUT_F32) != 0;
    const void* dpos = pos;
    const void* dq = q;
    if ((flags & RBE2D_HOST_BUFFERS) && N > 0) {
        r = stage_inputs(c, N, pos, q, in_f32, &dpos, &dq);
        if (r) return r;
    }
    r = run_sf(c, N, dpos, dq, in_f32, true);
    if (r) return r;
    if (rho_out) {
        cudaMemcpyKind kind = (flags & RBE2D_HOST_BUFFERS) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        CK(cudaMemcpyAsync(rho_out, c->rs, sizeof(double) * 4 * c->dp.P, kind, c->st), "copy structure factors");
    }
    if (flags & RBE2D_HOST_BUFFERS) CK(cudaStreamSynchronize(c->st), "synchronise");
    if (flags & RBE2D_VALIDATE) return validate(c);
    return RBE2D_OK;
}

int rbe2d_force(rbe2d_ctx* c, int64_t N, const void* pos, const void* q, int flags, void* force_out, void* phi_out,
                double* energy_out) {
    int r = check_common(c, N, pos, q);
    if (r) return r;
    if ((flags & RBE2D_REAL) && !c->real)
        return fail(c, RBE2D_EINVAL, "RBE2D_REAL needs a context created with real_space = 1");
    if (N > 0 && !force_out) return fail(c, RBE2D_EINVAL, "force_out must not be NULL");
    if ((flags & RBE2D_ACCUMULATE) && (flags & RBE2D_HOST_BUFFERS))
        return fail(c, RBE2D_EINVAL, "RBE2D_ACCUMULATE works on device buffers only");
    DeviceGuard g(c->device);
    const bool host = (flags & RBE2D_HOST_BUFFERS) != 0;
    const bool in_f32 = (flags & RBE2D_INPUT_F32) != 0;
    const void* dpos = pos;
    const void* dq = q;
    // host buffers in pinned memory: the kernels read the inputs and write the outputs in
    // place, so the transfers overlap the computation; other host memory is staged
    bool zero_copy = false;
    void *zf = nullptr, *zp = nullptr;
    if (host && N > 0) {
        const void* vp = device_view(pos);
        const void* vq = device_view(q);
        zf = device_view(force_out);
        zp = (flags & RBE2D_POTENTIAL) ? device_view(phi_out) : nullptr;
        zero_copy = vp && vq && zf && (zp || !(flags & RBE2D_POTENTIAL));
        if (zero_copy) {
            dpos = vp;
            dq = vq;
        } else {
            r = stage_inputs(c, N, pos, q, in_f32, &dpos, &dq);
            if (r) return r;
        }
    }
    const bool need_sigma = c->dp.diel != 0;
    const bool reuse = (flags & RBE2D_REUSE_SF) && c->sf_valid && c->sf_N == N && (c->sf_sigma || !need_sigma);
    // a real-space-only call needs no structure factor: the force starts from zero
    const bool real_only = !(flags & (RBE2D_KSPACE | RBE2D_IBC | RBE2D_ENERGY | RBE2D_POTENTIAL | RBE2D_VALIDATE));
    if (!reuse && !real_only) {
        r = run_sf(c, N, dpos, dq, in_f32, need_sigma, zero_copy);
        if (r) return r;
    }
    const size_t es = c->fp64 ? sizeof(double) : sizeof(float);
    void* fdev = zero_copy ? zf : (host ? c->stage_out : force_out);
    void* pdev = (flags & RBE2D_POTENTIAL) ? (zero_copy ? zp : (host ? c->stage_out2 : phi_out)) : nullptr;
    if ((flags & RBE2D_POTENTIAL) && !phi_out) return fail(c, RBE2D_EINVAL, "RBE2D_POTENTIAL needs phi_out");
    if (N > 0 && real_only) {
        if (!(flags & RBE2D_ACCUMULATE))
            CK(cudaMemsetAsync(fdev, 0, (size_t)N * 3 * es, c->st), "clear force");
    } else if (N > 0) {
        KTimer kt(c, RBE2D_TIMER_FORCE);
        CK(launch_force(c->st, c->dp, N, c->part, c->fp64, c->krec, c->scal, flags, fdev, pdev, 1.0, 1.0, c->sh,
                        c->counters, force_poly(c, pdev), force_shape(c, pdev)),
           "force launch");
    }
    if (flags & RBE2D_REAL) {
        KTimer kt(c, RBE2D_TIMER_REAL);
        CK(launch_real(c->st, c->dp, c->grid, c->rb, N, dpos, dq, in_f32, c->fp64, fdev, pdev,
                       (flags & RBE2D_POTENTIAL) ? 1 : 0, (flags & RBE2D_ENERGY) ? 1 : 0, c->scal, c->counters + 3,
                       c->status),
           "real-space launch");
        c->ureal_set = true;
    } else if (c->ureal_set) {
        CK(cudaMemsetAsync(c->scal + SC_UREAL, 0, sizeof(double), c->st), "clear real-space energy");
        c->ureal_set = false;
    }
    if ((flags & RBE2D_ENERGY) && energy_out) {
        if (host) CK(cudaMemcpyAsync(energy_out, c->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->st), "copy energy");
        else CK(launch_copy_energy(c->st, c->scal, energy_out), "copy energy");
    }
    if (host) {
        if (!zero_copy) {
            if (N > 0)
                CK(cudaMemcpyAsync(force_out, fdev, (size_t)N * 3 * es, cudaMemcpyDeviceToHost, c->st), "copy force");
            if (pdev && N > 0)
                CK(cudaMemcpyAsync(phi_out, pdev, (size_t)N * es, cudaMemcpyDeviceToHost, c->st), "copy phi");
        }
        CK(cudaStreamSynchronize(c->st), "synchronise");
    }
    if (flags & RBE2D_VALIDATE) return validate(c);
    return RBE2D_OK;
}

int rbe2d_force_lattice(rbe2d_ctx* c, int64_t N, const void* pos, const void* q, int flags, const int32_t* nmax,
                        void* force_out, void* phi_out, double* energy_out) {
    if (!c) return RBE2D_EINVAL;
    if (N < 0 || N > c->n_max) return fail(c, RBE2D_EINVAL, "N = %lld outside [0, n_max = %lld]", (long long)N, (long long)c->n_max);
    if (N > 0 && (!pos || !q || !force_out)) return fail(c, RBE2D_EINVAL, "pos, q and force_out must not be NULL");
    const int allowed = RBE2D_KSPACE | RBE2D_IBC | RBE2D_ENERGY | RBE2D_POTENTIAL | RBE2D_INPUT_F32 | RBE2D_ACCUMULATE;
    if (flags & ~allowed) return fail(c, RBE2D_EINVAL, "rbe2d_force_lattice accepts KSPACE, IBC, ENERGY, POTENTIAL, INPUT_F32, ACCUMULATE");
    if ((flags & RBE2D_POTENTIAL) && N > 0 && !phi_out) return fail(c, RBE2D_EINVAL, "RBE2D_POTENTIAL needs phi_out");
    if (!nmax) return fail(c, RBE2D_EINVAL, "nmax must not be NULL");
    int nm[3];
    for (int d = 0; d < 3; d++) {
        if (nmax[d] < 0 || nmax[d] > (1 << 20)) return fail(c, RBE2D_EINVAL, "nmax[%d] = %d outside [0, 2^20]", d, nmax[d]);
        nm[d] = nmax[d];
    }
    const double box = (2.0 * nm[0] + 1) * (2.0 * nm[1] + 1) * (2.0 * nm[2] + 1);
    if (box > 9.0e15) return fail(c, RBE2D_EINVAL, "the lattice box has more than 9e15 points");
    const int64_t n_half = ((int64_t)(2 * nm[0] + 1) * (2 * nm[1] + 1) * (2 * nm[2] + 1) - 1) / 2;
    if (n_half == 0) return fail(c, RBE2D_EINVAL, "the lattice box holds no k != 0");
    DeviceGuard g(c->device);
    const bool in_f32 = (flags & RBE2D_INPUT_F32) != 0;
    const int64_t P = c->dp.P, nchunks = (n_half + P - 1) / P;
    for (int64_t ch = 0; ch < nchunks; ch++) {
        {
            KTimer kt(c, RBE2D_TIMER_SAMPLE);
            CK(launch_lattice_k(c->st, c->dp, nm, ch * P, n_half, c->kc), "lattice batch launch");
        }
        c->have_batch = true;
        int r = run_sf(c, N, pos, q, in_f32, c->dp.diel != 0);
        if (r) return r;
        CK(launch_accum_uk(c->st, c->scal, ch == 0, ch == nchunks - 1), "energy accumulation");
        if (N > 0) {
            // the first chunk carries the IBC and self terms and honours RBE2D_ACCUMULATE;
            // later chunks add their k-space part only
            int fl = RBE2D_KSPACE | (flags & RBE2D_POTENTIAL);
            fl |= ch == 0 ? (flags & (RBE2D_IBC | RBE2D_ACCUMULATE)) : (RBE2D_ACCUMULATE | kForceNoSelf);
            KTimer kt(c, RBE2D_TIMER_FORCE);
            void* phi = (flags & RBE2D_POTENTIAL) ? phi_out : nullptr;
            CK(launch_force(c->st, c->dp, N, c->part, c->fp64, c->krec, c->scal, fl, force_out, phi, 1.0, 1.0, c->sh,
                            c->counters, force_poly(c, phi), force_shape(c, phi)),
               "force launch");
        }
    }
    c->ureal_set = false;
    if ((flags & RBE2D_ENERGY) && energy_out) CK(launch_copy_energy(c->st, c->scal, energy_out), "copy energy");
    return RBE2D_OK;
}

int rbe2d_energy_backward(rbe2d_ctx* c, int64_t N, const void* pos, const void* q, int flags, double grad_energy,
                          void* dpos_out, void* dq_out, double* dgamma) {
    int r = check_common(c, N, pos, q);
    if (r) return r;
    DeviceGuard g(c->device);
    const bool in_f32 = (flags & RBE2D_INPUT_F32) != 0;
    const bool need_sigma = c->dp.diel != 0;
    const bool reuse = (flags & RBE2D_REUSE_SF) && c->sf_valid && c->sf_N == N && (c->sf_sigma || !need_sigma);
    if (!reuse) {
        r = run_sf(c, N, pos, q, in_f32, need_sigma);
        if (r) return r;
    }
    if (N > 0 && (dpos_out || dq_out)) {
        void* fdev = dpos_out ? dpos_out : c->stage_out;
        int fl = RBE2D_KSPACE | RBE2D_IBC | (dq_out ? RBE2D_POTENTIAL : 0);
        KTimer kt(c, RBE2D_TIMER_FORCE);
        CK(launch_force(c->st, c->dp, N, c->part, c->fp64, c->krec, c->scal, fl, fdev, dq_out, -grad_energy,
                        grad_energy, c->sh, c->counters, force_poly(c, dq_out), force_shape(c, dq_out)),
           "adjoint launch");
    }
    if (dgamma) CK(launch_dgamma(c->st, c->scal, grad_energy, dgamma), "dgamma launch");
    return RBE2D_OK;
}

int rbe2d_md_step(rbe2d_ctx* c, int64_t N, double* pos, double* vel, const double* q, void* force_inout,
                  uint64_t* step_dev, const rbe2d_md_params* md, int mode, double* stats_dev) {
    if (!c) return RBE2D_EINVAL;
    if (!md || !step_dev || N < 0 || N > c->n_max) return fail(c, RBE2D_EINVAL, "bad MD arguments");
    if (N > 0 && (!pos || !vel || !q || !force_inout)) return fail(c, RBE2D_EINVAL, "NULL MD array");
    if (!(md->dt > 0) || !(md->mass > 0) || !(md->kT >= 0) || !(md->gamma >= 0))
        return fail(c, RBE2D_EINVAL, "dt and mass must be positive, kT and gamma non-negative");
    const bool lj = md->sigma_lj > 0 && md->eps_lj != 0;
    if (lj && 1.122462048309373 * md->sigma_lj > c->dp.r_c)
        return fail(c, RBE2D_EINVAL, "the WCA cutoff 2^(1/6) sigma_lj exceeds r_c");
    if ((lj || (md->force_flags & RBE2D_REAL)) && !c->real)
        return fail(c, RBE2D_EINVAL, "WCA pairs and RBE2D_REAL need a context created with real_space = 1");
    DeviceGuard g(c->device);
    MdParams mp;
    mp.dt = md->dt; mp.gamma = md->gamma; mp.kT = md->kT; mp.mass = md->mass;
    mp.sigma_lj = md->sigma_lj; mp.eps_lj = md->eps_lj; mp.sigma_wall = md->sigma_wall; mp.eps_wall = md->eps_wall;
    mp.noise_seed = md->noise_seed;
    mp.hk = 0.5 * md->dt / md->mass;
    mp.hd = 0.5 * md->dt;
    mp.c1 = exp(-md->gamma * md->dt);
    mp.c2s = sqrt(fmax(0.0, 1.0 - mp.c1 * mp.c1)) * sqrt(md->kT / md->mass);
    mp.w_sig = (float)md->sigma_wall;
    mp.w_rcut = (float)(1.122462048309373 * md->sigma_wall);
    mp.w_f = (float)(24.0 * md->eps_wall);
    mp.w_sig_d = md->sigma_wall;
    mp.w_rcut_d = 1.122462048309373 * md->sigma_wall;
    mp.w_f_d = 24.0 * md->eps_wall;
    // heights out of both walls' reach, with a margin for the float32 rounding of z and H
    // (an empty range when the slab is thinner than two reaches; everything without walls)
    if (md->sigma_wall > 0) {
        const double margin = 1e-5 * (c->dp.H + mp.w_rcut_d) + 1e-12;
        mp.w_in_lo = mp.w_rcut_d + margin;
        mp.w_in_hi = fmax(mp.w_in_lo, c->dp.H - mp.w_rcut_d - margin);
    } else {
        mp.w_in_lo = 0.0;
        mp.w_in_hi = INFINITY;
    }
    const bool f64 = c->fp64;
    unsigned long long* step = (unsigned long long*)step_dev;
    if (mode & RBE2D_MD_STEP) {
        KTimer kt(c, RBE2D_TIMER_MD);
        CK(launch_md_baoa(c->st, c->dp, mp, N, pos, vel, force_inout, f64, step, c->status), "MD drift launch");
    }
    // force at the (new) positions: batch for this step, k-space, IBC, real space + WCA
    {
        KTimer kt(c, RBE2D_TIMER_SAMPLE);
        CK(launch_sample(c->st, c->dp, c->tables, c->p.seed, 0, step, c->kc, nullptr, c->status), "sample launch");
    }
    c->have_batch = true;
    int r = run_sf(c, N, pos, q, false, c->dp.diel != 0);
    if (r) return r;
    const int fl = md->force_flags & (RBE2D_KSPACE | RBE2D_IBC);
    if (N > 0) {
        KTimer kt(c, RBE2D_TIMER_FORCE);
        CK(launch_force(c->st, c->dp, N, c->part, c->fp64, c->krec, c->scal, fl, force_inout, nullptr, 1.0, 1.0,
                        c->sh, c->counters, c->f_poly, c->f_shape),
           "force launch");
    }
    if ((md->force_flags & RBE2D_REAL) || lj) {
        DevParams d = c->dp;
        if (lj) {
            d.lj_sig2 = md->sigma_lj * md->sigma_lj;
            d.lj_eps = md->eps_lj;
            d.lj_rc2 = 1.2599210498948732 * d.lj_sig2;  // (2^(1/6) sigma)^2
        }
        if (!(md->force_flags & RBE2D_REAL)) d.kc = 0.0;  // WCA only: the screened Coulomb term is off
        KTimer kt(c, RBE2D_TIMER_REAL);
        if (c->lists) {
            if (N != c->nl_N) CK(cudaMemsetAsync(c->nl.flag, 1, sizeof(int), c->st), "list rebuild flag");
            c->nl_N = N;
            CK(launch_real_lists(c->st, d, c->nl, c->rb, N, pos, q, (float*)force_inout, c->status),
               "real-space list launch");
        } else {
            CK(launch_real(c->st, d, c->grid, c->rb, N, pos, q, false, c->fp64, force_inout, nullptr, 0, 0, c->scal,
                           c->counters + 3, c->status),
               "real-space launch");
        }
        c->ureal_set = true;
    }
    if (mode & RBE2D_MD_STEP) {
        KTimer kt(c, RBE2D_TIMER_MD);
        CK(launch_md_b(c->st, c->dp, mp, N, pos, vel, force_inout, f64, step, c->md_kpart, stats_dev,
                       c->counters + 4),
           "MD kick launch");
    }
    return RBE2D_OK;
}

int rbe2d_md_list_stats(rbe2d_ctx* c, int* enabled_out, uint64_t* builds_out) {
    if (!c) return RBE2D_EINVAL;
    DeviceGuard g(c->device);
    unsigned long long b = 0;
    if (c->lists) {
        CK(cudaMemcpyAsync(&b, c->nl.builds, sizeof b, cudaMemcpyDeviceToHost, c->st), "read list builds");
    }
    CK(cudaStreamSynchronize(c->st), "synchronise");
    if (enabled_out) *enabled_out = c->lists ? 1 : 0;
    if (builds_out) *builds_out = b;
    return RBE2D_OK;
}

int rbe2d_autotune(rbe2d_ctx* c, int64_t N, const void* pos, const void* q, int flags, void* force_scratch,
                   int* choice) {
    int r = check_common(c, N, pos, q);
    if (r) return r;
    if (!force_scratch) return fail(c, RBE2D_EINVAL, "force_scratch must not be NULL");
    DeviceGuard g(c->device);
    int best[4] = {c->sf_poly, c->f_poly, c->sf_shape, c->f_shape};
    if (!c->fp64 && N > 0) {
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0), "event");
        CK(cudaEventCreate(&e1), "event");
        const int fl = (flags & (RBE2D_IBC | RBE2D_INPUT_F32)) | RBE2D_KSPACE;
        const bool in_f32 = (fl & RBE2D_INPUT_F32) != 0;
        // mean of three timed repetitions after one warm-up; which = 0: structure factor,
        // 1: force on the structure factors of the last structure-factor run
        auto time_it = [&](int which, float* ms_out) -> int {
            float tot = 0.f;
            for (int rep = 0; rep < 4; rep++) {
                CK(cudaEventRecord(e0, c->st), "event");
                int rr = which == 0 ? run_sf(c, N, pos, q, in_f32, c->dp.diel != 0)
                                    : rbe2d_force(c, N, pos, q, fl | RBE2D_REUSE_SF, force_scratch, nullptr, nullptr);
                if (rr) return rr;
                CK(cudaEventRecord(e1, c->st), "event");
                CK(cudaEventSynchronize(e1), "event");
                float a = 0.f;
                cudaEventElapsedTime(&a, e0, e1);
                if (rep > 0) tot += a;
            }
            *ms_out = tot / 3.f;
            return RBE2D_OK;
        };
        // structure factor: FMA-pipe share x shape
        float best_ms = 1e30f;
        for (int v = 0; v < kPolyLevels; v++)
            for (int a = 0; a < kSfShapes; a++) {
                c->sf_poly = v;
                c->sf_shape = a;
                float ms = 0.f;
                r = time_it(0, &ms);
                if (r) return r;
                if (ms < best_ms) { best_ms = ms; best[0] = v; best[2] = a; }
            }
        c->sf_poly = best[0];
        c->sf_shape = best[2];
        r = run_sf(c, N, pos, q, in_f32, c->dp.diel != 0);
        if (r) return r;
        // force: FMA-pipe share x shape
        best_ms = 1e30f;
        for (int v = 0; v < kPolyLevels; v++)
            for (int b = 0; b < kForceShapes; b++) {
                c->f_poly = v;
                c->f_shape = b;
                float ms = 0.f;
                r = time_it(1, &ms);
                if (r) return r;
                if (ms < best_ms) { best_ms = ms; best[1] = v; best[3] = b; }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    c->sf_poly = best[0];
    c->f_poly = best[1];
    c->sf_shape = best[2];
    c->f_shape = best[3];
    c->sf_valid = false;
    if (choice)
        for (int i = 0; i < 4; i++) choice[i] = best[i];
    return RBE2D_OK;
}

int rbe2d_autotune_potential(rbe2d_ctx* c, int64_t N, const void* pos, const void* q, int flags,
                             void* force_scratch, void* phi_scratch, int* choice) {
    int r = check_common(c, N, pos, q);
    if (r) return r;
    if (!force_scratch || !phi_scratch) return fail(c, RBE2D_EINVAL, "force_scratch and phi_scratch must not be NULL");
    DeviceGuard g(c->device);
    int best[2] = {c->p_poly, c->p_shape};
    if (!c->fp64 && N > 0) {
        const int fl = (flags & (RBE2D_IBC | RBE2D_INPUT_F32)) | RBE2D_KSPACE | RBE2D_POTENTIAL | RBE2D_REUSE_SF;
        r = run_sf(c, N, pos, q, (fl & RBE2D_INPUT_F32) != 0, c->dp.diel != 0);
        if (r) return r;
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0), "event");
        CK(cudaEventCreate(&e1), "event");
        // mean of three timed repetitions after one warm-up
        float best_ms = 1e30f;
        for (int v = 0; v < kPolyLevels && !r; v++)
            for (int b = 0; b < kPotShapes && !r; b++) {
                c->p_poly = v;
                c->p_shape = b;
                float tot = 0.f;
                for (int rep = 0; rep < 4 && !r; rep++) {
                    CK(cudaEventRecord(e0, c->st), "event");
                    r = rbe2d_force(c, N, pos, q, fl, force_scratch, phi_scratch, nullptr);
                    CK(cudaEventRecord(e1, c->st), "event");
                    CK(cudaEventSynchronize(e1), "event");
                    float a = 0.f;
                    cudaEventElapsedTime(&a, e0, e1);
                    if (rep > 0) tot += a;
                }
                if (!r && tot / 3.f < best_ms) { best_ms = tot / 3.f; best[0] = v; best[1] = b; }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (r) return r;
    }
    c->p_poly = best[0];
    c->p_shape = best[1];
    if (choice) { choice[0] = best[0]; choice[1] = best[1]; }
    return RBE2D_OK;
}

int rbe2d_set_tuning_potential(rbe2d_ctx* c, const int* choice) {
    if (!c) return RBE2D_EINVAL;
    if (!choice || choice[0] < 0 || choice[0] > kPolyLevels - 1 || choice[1] < 0 || choice[1] >= kPotShapes)
        return fail(c, RBE2D_EINVAL, "potential tuning choice must be {0..%d, 0..%d}", kPolyLevels - 1, kPotShapes - 1);
    c->p_poly = choice[0];
    c->p_shape = choice[1];
    return RBE2D_OK;
}

int rbe2d_set_tuning(rbe2d_ctx* c, const int* choice) {
    if (!c) return RBE2D_EINVAL;
    if (!choice || choice[0] < 0 || choice[0] > kPolyLevels - 1 || choice[1] < 0 || choice[1] > kPolyLevels - 1 ||
        choice[2] < 0 || choice[2] >= kSfShapes || choice[3] < 0 || choice[3] >= kForceShapes)
        return fail(c, RBE2D_EINVAL, "tuning choice must be {0..%d, 0..%d, 0..%d, 0..%d}", kPolyLevels - 1,
                    kPolyLevels - 1, kSfShapes - 1, kForceShapes - 1);
    c->sf_poly = choice[0];
    c->f_poly = choice[1];
    c->sf_shape = choice[2];
    c->f_shape = choice[3];
    c->sf_valid = false;
    return RBE2D_OK;
}

int rbe2d_charge_sums(rbe2d_ctx* c, double* sums_out) {
    if (!c || !sums_out) return c ? fail(c, RBE2D_EINVAL, "sums_out must not be NULL") : RBE2D_EINVAL;
    if (!c->sf_valid) return fail(c, RBE2D_EINVAL, "no structure factor evaluated yet");
    DeviceGuard g(c->device);
    CK(launch_copy_sums(c->st, c->scal, sums_out), "copy charge sums");
    return RBE2D_OK;
}

int rbe2d_set_structure_factor(rbe2d_ctx* c, int64_t N, const double* rho, const double* sums) {
    if (!c) return RBE2D_EINVAL;
    if (!rho || !sums) return fail(c, RBE2D_EINVAL, "rho and sums must not be NULL");
    if (!c->have_batch) return fail(c, RBE2D_EINVAL, "no k batch: call rbe2d_sample_k or rbe2d_set_k first");
    if (!c->sf_valid || c->sf_N != N)
        return fail(c, RBE2D_EINVAL, "call rbe2d_structure_factor on the local particles (same N) first");
    DeviceGuard g(c->device);
    CK(launch_inject_totals(c->st, c->dp.P, rho, sums, c->sf_part, c->pack_part), "inject totals");
    {
        KTimer kt(c, RBE2D_TIMER_FOLD);
        CK(launch_fold(c->st, c->dp, c->sf_part, 1, c->kc, c->fp64, c->rs, c->kterm, c->krec, c->pack_part, 1,
                       c->pack2, c->scal, c->counters),
           "fold launch");
    }
    c->sf_sigma = 1;
    c->ureal_set = false;
    return RBE2D_OK;
}

int rbe2d_timer_enable(rbe2d_ctx* c, int capacity, unsigned class_mask) {
    if (!c) return RBE2D_EINVAL;
    if (capacity < 0 || capacity > (1 << 20)) return fail(c, RBE2D_EINVAL, "timer capacity outside [0, 2^20]");
    if (class_mask >> RBE2D_TIMER_COUNT) return fail(c, RBE2D_EINVAL, "timer class mask has unknown bits");
    DeviceGuard g(c->device);
    CK(cudaStreamSynchronize(c->st), "synchronise");
    timer_free(c);
    if (capacity == 0) return RBE2D_OK;
    for (int k = 0; k < RBE2D_TIMER_COUNT; k++) {
        if (!(class_mask >> k & 1u)) continue;
        c->tev[k].resize(2 * (size_t)capacity, nullptr);
        for (auto& e : c->tev[k]) {
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) {
                e = nullptr;
                for (int j = 0; j <= k; j++) {
                    for (cudaEvent_t x : c->tev[j])
                        if (x) cudaEventDestroy(x);
                    c->tev[j].clear();
                }
                return cuda_fail(c, err, "create timer events");
            }
        }
    }
    c->tcap = capacity;
    c->tmask = class_mask;
    return RBE2D_OK;
}

int rbe2d_timer_read(rbe2d_ctx* c, double* total_ms, int64_t* launches) {
    if (!c) return RBE2D_EINVAL;
    if (!total_ms) return fail(c, RBE2D_EINVAL, "total_ms must not be NULL");
    DeviceGuard g(c->device);
    CK(cudaStreamSynchronize(c->st), "synchronise");
    for (int k = 0; k < RBE2D_TIMER_COUNT; k++) {
        double t = 0.0;
        for (int i = 0; i < c->tn[k]; i++) {
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, c->tev[k][2 * i], c->tev[k][2 * i + 1]), "read timer events");
            t += ms;
        }
        total_ms[k] = t;
        if (launches) launches[k] = c->tn[k];
        c->tn[k] = 0;
    }
    return RBE2D_OK;
}

int rbe2d_kernel_launches(uint64_t* count_out) {
    if (!count_out) return RBE2D_EINVAL;
    *count_out = g_kernel_launches.load(std::memory_order_relaxed);
    return RBE2D_OK;
}

int rbe2d_sync_status(rbe2d_ctx* c) {
    if (!c) return RBE2D_EINVAL;
    DeviceGuard g(c->device);
    int s[ST_COUNT];
    CK(cudaStreamSynchronize(c->st), "synchronise");
    CK(cudaMemcpy(s, c->status, sizeof s, cudaMemcpyDeviceToHost), "read status");
    CK(cudaMemset(c->status, 0, sizeof s), "clear status");
    if (s[ST_SAMPLER]) return fail(c, RBE2D_ESAMPLER, "%d k-samples were rejected 64 times (or were k = 0)", s[ST_SAMPLER]);
    if (s[ST_TIMEOUT]) return fail(c, RBE2D_ETIMEOUT, "a bounded device wait gave up (%d)", s[ST_TIMEOUT]);
    if (s[ST_CELL])
        return fail(c, RBE2D_ERANGE, "real-space cell list over its work limits %d times (crowded cells)", s[ST_CELL]);
    if (s[ST_MD]) return fail(c, RBE2D_ERANGE, "%d MD particle updates were not finite", s[ST_MD]);
    return RBE2D_OK;
}

}  // extern "C"
