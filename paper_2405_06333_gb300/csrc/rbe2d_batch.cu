// C ABI of the batched launch (include/rbe2d.h, rbe2d_batch_*): many independent slab
// systems, each with its own geometry, contrasts, image levels and batch, evaluated by
// one sampling launch and one persistent launch (batch_kernels.cu).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>

#include <string>
#include <vector>

#include "rbe2d_internal.h"
#include "rbe2d_setup.h"

using namespace rbe2d;

struct rbe2d_batch {
    int n_sys = 0, P_max = 0, device = 0;
    cudaStream_t st = nullptr;
    std::vector<BatchSys> host_sys;
    std::vector<int64_t> off;
    int64_t n_total = 0;
    // device
    BatchSys* sys = nullptr;
    int* item_sys = nullptr;
    double* cdf = nullptr;
    int* guide = nullptr;
    KCoef* kc = nullptr;
    double* eo = nullptr;
    KPair32* krec = nullptr;
    uint4* part = nullptr;
    double* partial = nullptr;
    double* pack = nullptr;
    double* scal = nullptr;
    int* sf_done = nullptr;
    int* ready = nullptr;
    int* head = nullptr;
    unsigned* exit_count = nullptr;
    int* status = nullptr;
    int64_t items_cap = 0, partial_cap = 0;
    // launch shape
    int sf_chunk = 512, f_chunk = 256, grid = 0, sms = 1;
    int variant = 0, occ[2] = {1, 1};  // kernel variant (bit 0: register cap, bit 1: FMA-pipe angles), CTAs per SM by bit 0
    int n_sf_items = 0, n_f_items = 0;
    // bounded wait of the force items and the system kept unpublished (timeout tests)
    unsigned long long wait_ns = 2000000000ull;
    int withhold = -1;
    std::string err;
};

namespace {

int bfail(rbe2d_batch* b, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return code;
}

#define BCK(call, where)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return bfail(b, RBE2D_ECUDA, "%s: %s", where, cudaGetErrorString(e_)); \
    } while (0)

void bfree(rbe2d_batch* b) {
    cudaFree(b->sys); cudaFree(b->item_sys); cudaFree(b->cdf); cudaFree(b->guide); cudaFree(b->kc); cudaFree(b->eo);
    cudaFree(b->krec); cudaFree(b->part); cudaFree(b->partial); cudaFree(b->pack); cudaFree(b->scal); cudaFree(b->sf_done);
    cudaFree(b->ready); cudaFree(b->head); cudaFree(b->exit_count); cudaFree(b->status);
}

// Work items for the chunk sizes: per system ceil(N / chunk) (at least one), structure-
// factor items first.  Fills the host records and uploads them with the item map.
int build_items(rbe2d_batch* b, int sf_chunk, int f_chunk) {
    std::vector<int> items;
    int sf = 0;
    int64_t part = 0;
    for (int s = 0; s < b->n_sys; s++) {
        BatchSys& bs = b->host_sys[s];
        bs.nsf = (int)std::max<int64_t>(1, (bs.N + sf_chunk - 1) / sf_chunk);
        bs.sf_base = sf;
        bs.part_base = part;
        part += (int64_t)bs.dp.P * bs.nsf * 4;
        sf += bs.nsf;
        for (int i = 0; i < bs.nsf; i++) items.push_back(s);
    }
    int f = 0;
    for (int s = 0; s < b->n_sys; s++) {
        BatchSys& bs = b->host_sys[s];
        bs.nf = (int)std::max<int64_t>(1, (bs.N + f_chunk - 1) / f_chunk);
        bs.f_base = f;
        f += bs.nf;
        for (int i = 0; i < bs.nf; i++) items.push_back(s);
    }
    if ((int64_t)items.size() > b->items_cap || part > b->partial_cap)
        return bfail(b, RBE2D_EINVAL, "chunk sizes below the minimum the batch was sized for");
    b->n_sf_items = sf;
    b->n_f_items = f;
    b->sf_chunk = sf_chunk;
    b->f_chunk = f_chunk;
    BCK(cudaMemcpy(b->sys, b->host_sys.data(), sizeof(BatchSys) * b->n_sys, cudaMemcpyHostToDevice), "upload systems");
    BCK(cudaMemcpy(b->item_sys, items.data(), sizeof(int) * items.size(), cudaMemcpyHostToDevice), "upload items");
    return RBE2D_OK;
}

BatchArgs args_of(rbe2d_batch* b, const double* pos, const double* q, float* force, int ibc) {
    BatchArgs a;
    a.sys = b->sys; a.n_sys = b->n_sys; a.P_max = b->P_max;
    a.item_sys = b->item_sys; a.n_sf_items = b->n_sf_items; a.n_f_items = b->n_f_items;
    a.sf_chunk = b->sf_chunk; a.f_chunk = b->f_chunk;
    a.pos = pos; a.q = q; a.force = force; a.ibc = ibc;
    a.kc = b->kc; a.eo = b->eo; a.krec = b->krec; a.KP = (b->P_max + 1) / 2; a.part = b->part; a.partial = b->partial; a.pack = b->pack; a.scal = b->scal;
    a.sf_done = b->sf_done; a.ready = b->ready; a.head = b->head; a.exit_count = b->exit_count; a.status = b->status;
    a.wait_ns = b->wait_ns;
    a.withhold = b->withhold;
    return a;
}

constexpr int kMinSfChunk = 256, kMinFChunk = 256;

}  // namespace

extern "C" {

int rbe2d_batch_init(const rbe2d_params* per_sys, int n_sys, const int64_t* offsets, void* stream,
                     rbe2d_batch** out) {
    if (!out) return RBE2D_EINVAL;
    *out = nullptr;
    if (!per_sys || !offsets || n_sys < 1) return RBE2D_EINVAL;
    rbe2d_batch* b = new (std::nothrow) rbe2d_batch();
    if (!b) return RBE2D_ENOMEM;
    b->n_sys = n_sys;
    b->st = (cudaStream_t)stream;
    cudaGetDevice(&b->device);
    std::vector<double> cdf_all;
    std::vector<int> guide_all;
    long long eo_total = 0;  // float64 entries of the per-kz image-series tables
    for (int s = 0; s < n_sys; s++) {
        rbe2d_params p = per_sys[s];
        const int64_t N = offsets[s + 1] - offsets[s];
        if (N < 0 || !(p.Lx > 0) || !(p.Ly > 0) || !(p.H > 0) || !(fabs(p.gamma_top) <= 1) ||
            !(fabs(p.gamma_bot) <= 1) || p.P < 1 || p.P > 128 * kBatchKR || p.precision != RBE2D_FP32_MIXED) {
            delete b;
            return RBE2D_EINVAL;
        }
        if (!(p.eps > 0)) p.eps = 1e-4;
        if (!(p.coulomb_k > 0)) p.coulomb_k = 1.0;
        if (!(p.alpha > 0)) p.alpha = cbrt((double)(N > 0 ? N : 1) / (p.Lx * p.Ly * p.H));
        if (p.M < 0) p.M = auto_M(p.Lx, p.Ly, p.H, p.gamma_top, p.gamma_bot, p.eps);
        if (!(p.Lz > 0)) p.Lz = auto_Lz(p.Lx, p.Ly, p.H, p.M, p.alpha, p.eps);
        if (p.Lz < (p.M + 1) * p.H) { delete b; return RBE2D_EINVAL; }
        BatchSys bs = {};
        DevParams& dp = bs.dp;
        std::vector<double> cdf[3];
        double Sd[3];
        const double Ls[3] = {p.Lx, p.Ly, p.Lz};
        for (int d = 0; d < 3; d++) {
            Sd[d] = build_cdf(p.alpha, Ls[d], &cdf[d]);
            std::vector<int> gd;
            build_guide(cdf[d], &gd);
            bs.tab_off[d] = (int)cdf_all.size();
            bs.tab_len[d] = (int)cdf[d].size();
            cdf_all.insert(cdf_all.end(), cdf[d].begin(), cdf[d].end());
            guide_all.insert(guide_all.end(), gd.begin(), gd.end());
        }
        ImageConsts ic;
        image_constants(p.gamma_top, p.gamma_bot, p.M, &ic);
        dp.Lx = p.Lx; dp.Ly = p.Ly; dp.H = p.H; dp.Lz = p.Lz; dp.V = p.Lx * p.Ly * p.Lz;
        dp.inv_Lx = 1.0 / p.Lx; dp.inv_Ly = 1.0 / p.Ly; dp.inv_Lz = 1.0 / p.Lz;
        dp.S = Sd[0] * Sd[1] * Sd[2] - 1.0;
        dp.alpha = p.alpha; dp.r_c = p.r_c > 0 ? p.r_c : 3.0 / p.alpha;
        dp.gt = p.gamma_top; dp.gb = p.gamma_bot; dp.kc = p.coulomb_k;
        dp.coef = 2.0 * M_PI / dp.V * (dp.S / p.P) * p.coulomb_k;
        dp.cM = ic.cM; dp.dM = ic.dM; dp.dcM_t = ic.dcM_t; dp.dcM_b = ic.dcM_b; dp.ddM_t = ic.ddM_t; dp.ddM_b = ic.ddM_b;
        dp.M = p.M; dp.P = p.P; dp.P_pad = p.P;
        dp.diel = 1;  // the batched kernel always sums sigma (E = O = 0 reproduces the homogeneous case)
        dp.kseg = 4;  // lanes per kz in the table kernel
        while (dp.kseg < 32 && dp.kseg < p.M / 2 + 1) dp.kseg *= 2;
        bs.eo_half = bs.tab_len[2] / 2;  // every kz the sampler can draw
        bs.eo_off = eo_total;
        eo_total += 9LL * (2 * bs.eo_half + 1);
        bs.off = offsets[s];
        bs.N = N;
        bs.seed = p.seed;
        b->host_sys.push_back(bs);
        if (p.P > b->P_max) b->P_max = p.P;
        b->n_total = offsets[s + 1] > b->n_total ? offsets[s + 1] : b->n_total;
    }
    // capacity for the smallest chunk sizes the tuner may pick
    int64_t items = 0, part = 0;
    for (auto& bs : b->host_sys) {
        const int64_t nsf = std::max<int64_t>(1, (bs.N + kMinSfChunk - 1) / kMinSfChunk);
        const int64_t nf = std::max<int64_t>(1, (bs.N + kMinFChunk - 1) / kMinFChunk);
        items += nsf + nf;
        part += (int64_t)bs.dp.P * nsf * 4;
    }
    b->items_cap = items;
    b->partial_cap = part;
    bool ok = true;
    auto al = [&](void** p, size_t bytes) {
        if (ok && cudaMalloc(p, bytes < 16 ? 16 : bytes) != cudaSuccess) ok = false;
    };
    al((void**)&b->sys, sizeof(BatchSys) * n_sys);
    al((void**)&b->item_sys, sizeof(int) * (size_t)items);
    al((void**)&b->cdf, sizeof(double) * cdf_all.size());
    al((void**)&b->guide, sizeof(int) * guide_all.size());
    al((void**)&b->kc, sizeof(KCoef) * (size_t)n_sys * b->P_max);
    al((void**)&b->eo, sizeof(double) * (size_t)eo_total);
    al((void**)&b->krec, sizeof(KPair32) * (size_t)n_sys * ((b->P_max + 1) / 2));
    al((void**)&b->part, sizeof(uint4) * (size_t)(b->n_total > 0 ? b->n_total : 1));
    al((void**)&b->partial, sizeof(double) * (size_t)part);
    al((void**)&b->pack, sizeof(double) * 4 * (size_t)items);
    al((void**)&b->scal, sizeof(double) * 4 * (size_t)n_sys);
    al((void**)&b->sf_done, sizeof(int) * n_sys);
    al((void**)&b->ready, sizeof(int) * n_sys);
    al((void**)&b->head, sizeof(int));
    al((void**)&b->exit_count, sizeof(unsigned));
    al((void**)&b->status, sizeof(int) * ST_COUNT);
    if (!ok) {
        cudaGetLastError();
        bfree(b);
        delete b;
        return RBE2D_ENOMEM;
    }
    cudaError_t e = cudaMemcpy(b->cdf, cdf_all.data(), sizeof(double) * cdf_all.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->guide, guide_all.data(), sizeof(int) * guide_all.size(), cudaMemcpyHostToDevice);
    // the image-series sums of every kz of every system's sampler box, once
    for (int s = 0; s < n_sys && e == cudaSuccess; s++) {
        const BatchSys& bs = b->host_sys[s];
        e = launch_eo_table(0, bs.dp, bs.eo_half, b->eo + bs.eo_off);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemset(b->sf_done, 0, sizeof(int) * n_sys);
    if (e == cudaSuccess) e = cudaMemset(b->ready, 0, sizeof(int) * n_sys);
    if (e == cudaSuccess) e = cudaMemset(b->head, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->exit_count, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int) * ST_COUNT);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = batch_occupancy(b->P_max, 0, &b->occ[0]);
    if (e == cudaSuccess) e = batch_occupancy(b->P_max, 1, &b->occ[1]);
    if (e != cudaSuccess || build_items(b, 512, 256) != RBE2D_OK) {
        bfree(b);
        delete b;
        return RBE2D_ECUDA;
    }
    for (int v = 0; v < 2; v++)
        if (b->occ[v] < 1) b->occ[v] = 1;
    b->grid = b->sms * b->occ[0];
    *out = b;
    return RBE2D_OK;
}

int rbe2d_batch_destroy(rbe2d_batch* b) {
    if (!b) return RBE2D_OK;
    cudaStreamSynchronize(b->st);
    bfree(b);
    delete b;
    return RBE2D_OK;
}

const char* rbe2d_batch_last_error(const rbe2d_batch* b) { return b ? b->err.c_str() : "null batch"; }

int rbe2d_batch_force(rbe2d_batch* b, uint64_t step, const double* pos, const double* q, int flags, float* force_out,
                      double* energy_out) {
    if (!b) return RBE2D_EINVAL;
    if (b->n_total > 0 && (!pos || !q || !force_out)) return bfail(b, RBE2D_EINVAL, "NULL array");
    BatchArgs a = args_of(b, pos, q, force_out, (flags & RBE2D_IBC) ? 1 : 0);
    BCK(launch_batch_sample(b->st, a, b->cdf, b->guide, step), "batched sample launch");
    BCK(launch_batch(b->st, a, b->grid, b->variant), "batched persistent launch");
    if ((flags & RBE2D_ENERGY) && energy_out)
        BCK(cudaMemcpyAsync(energy_out, b->scal, sizeof(double) * 4 * b->n_sys, cudaMemcpyDeviceToDevice, b->st),
            "copy energies");
    return RBE2D_OK;
}

int rbe2d_batch_sync_status(rbe2d_batch* b) {
    if (!b) return RBE2D_EINVAL;
    int s[ST_COUNT];
    BCK(cudaStreamSynchronize(b->st), "synchronise");
    BCK(cudaMemcpy(s, b->status, sizeof s, cudaMemcpyDeviceToHost), "read status");
    BCK(cudaMemset(b->status, 0, sizeof s), "clear status");
    if (s[ST_SAMPLER]) return bfail(b, RBE2D_ESAMPLER, "%d k-samples were rejected 64 times", s[ST_SAMPLER]);
    if (s[ST_TIMEOUT]) return bfail(b, RBE2D_ETIMEOUT, "%d force items gave up waiting for their system", s[ST_TIMEOUT]);
    return RBE2D_OK;
}

int rbe2d_batch_set_wait(rbe2d_batch* b, double seconds, int withhold_sys) {
    if (!b) return RBE2D_EINVAL;
    if (!(seconds > 0.0) || !(seconds <= 10.0))
        return bfail(b, RBE2D_EINVAL, "wait limit %g s outside (0, 10]", seconds);
    if (withhold_sys < -1 || withhold_sys >= b->n_sys)
        return bfail(b, RBE2D_EINVAL, "withheld system %d outside [-1, %d)", withhold_sys, b->n_sys);
    b->wait_ns = (unsigned long long)(seconds * 1e9);
    if (b->wait_ns < 1) b->wait_ns = 1;
    b->withhold = withhold_sys;
    return RBE2D_OK;
}

int rbe2d_batch_set_tuning(rbe2d_batch* b, const int* choice) {
    if (!b) return RBE2D_EINVAL;
    if (!choice) return bfail(b, RBE2D_EINVAL, "choice must not be NULL");
    const int sc = choice[0], fc = choice[1], grid = choice[2], v = choice[3];
    if (sc < kMinSfChunk || fc < kMinFChunk || grid < 1 || v < 0 || v > 3 || ((v & 1) && b->P_max > 256))
        return bfail(b, RBE2D_EINVAL, "tuning choice out of range");
    const int r = build_items(b, sc, fc);
    if (r) return r;
    b->variant = v;
    b->grid = grid;
    return RBE2D_OK;
}

int rbe2d_batch_autotune(rbe2d_batch* b, const double* pos, const double* q, float* force_out, int* choice) {
    if (!b) return RBE2D_EINVAL;
    const int sf_c[] = {256, 512, 1024, 2048};
    const int f_c[] = {256, 512, 1024};
    const int mult[] = {1, 2};
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0), "event");
    BCK(cudaEventCreate(&e1), "event");
    float best = 1e30f;
    int bs_ = 512, bf = 256, bm = 1, bv = 0;
    for (int v = 0; v < 4; v++)
    for (int sc : sf_c)
        for (int fc : f_c)
            for (int m : mult) {
                if ((v & 1) && b->P_max > 256) continue;  // no register cap for 4 wave vectors per thread
                if (build_items(b, sc, fc) != RBE2D_OK) continue;
                b->variant = v;
                b->grid = b->sms * b->occ[v & 1] * m;
                float t = 0.f;
                for (int rep = 0; rep < 3; rep++) {
                    int r = rbe2d_batch_force(b, (uint64_t)rep, pos, q, RBE2D_KSPACE | RBE2D_IBC, force_out, nullptr);
                    if (r) return r;
                    if (rep == 0) continue;  // warm-up
                    BCK(cudaEventRecord(e0, b->st), "event");
                    r = rbe2d_batch_force(b, (uint64_t)rep, pos, q, RBE2D_KSPACE | RBE2D_IBC, force_out, nullptr);
                    if (r) return r;
                    BCK(cudaEventRecord(e1, b->st), "event");
                    BCK(cudaEventSynchronize(e1), "event");
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    t += ms;
                }
                if (t < best) { best = t; bs_ = sc; bf = fc; bm = m; bv = v; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int r = build_items(b, bs_, bf);
    if (r) return r;
    b->variant = bv;
    b->grid = b->sms * b->occ[bv & 1] * bm;
    if (choice) { choice[0] = bs_; choice[1] = bf; choice[2] = b->grid; choice[3] = bv; }
    return rbe2d_batch_sync_status(b);
}

}  // extern "C"
