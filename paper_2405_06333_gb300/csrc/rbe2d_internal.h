// Internal declarations shared by the host code and the kernels of librbe2d.
// Not part of the public ABI (include/rbe2d.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/rbe2d.h"

namespace rbe2d {

struct Shapes;

// Parameters handed to every kernel by value (all float64, computed once at init).
struct DevParams {
    double Lx, Ly, H, Lz, V;
    double inv_Lx, inv_Ly, inv_Lz;
    double S;          // sum_{k != 0} w(k) (Eq. 2.21)
    double alpha, r_c, gt, gb, kc;  // kc = coulomb_k
    double coef;       // (2 pi / V) (S / P) kc; c_l = -coef / k_l^2
    double cM, dM;     // U_IBC^M = (2pi/V) kc mu (cM mu + Q H dM)   (Eq. 3.18)
    double dcM_t, dcM_b, ddM_t, ddM_b;
    int M, P, P_pad;
    int diel;          // M > 0 and some gamma != 0
    int kseg;          // lanes per wave vector in the per-k kernels: power of two >= M/2 + 1, in [4, 32]
    // WCA pair repulsion between real charges inside the real-space pass (MD only;
    // lj_eps = 0: none): 4 eps [(s/r)^12 - (s/r)^6 + 1/4] for r < 2^(1/6) s
    double lj_sig2, lj_eps, lj_rc2;
    double coef_unit;  // (2 pi / V) kc: c = -coef_unit W / k^2 for a k with explicit weight W
    double self_c;     // -alpha kc / sqrt(pi): U_self = self_c sum q^2
    int acc;           // force kernels add their result to force / phi instead of storing it
};

// Langevin MD parameters (public rbe2d_md_params, copied for the kernels).
struct MdParams {
    double dt, gamma, kT, mass, sigma_lj, eps_lj, sigma_wall, eps_wall;
    unsigned long long noise_seed;
    // derived on the host: half kick per unit force dt/(2m), drift dt/2, O-step factors
    // c1 = exp(-gamma dt) and c2 sqrt(kT/m), c2 = sqrt(1 - c1^2); WCA wall constants
    double hk, hd, c1, c2s;
    float w_sig, w_rcut, w_f;  // wall sigma, 2^(1/6) sigma, 24 eps
    double w_sig_d, w_rcut_d, w_f_d;  // the same in float64 (float64 mode)
    double w_in_lo, w_in_hi;  // heights (>= 0) in [w_in_lo, w_in_hi) feel neither wall
};

cudaError_t launch_md_baoa(cudaStream_t st, const DevParams& dp, const MdParams& md, int64_t N, double* pos,
                           double* vel, const void* force, bool f64, const unsigned long long* step, int* status);
cudaError_t launch_md_b(cudaStream_t st, const DevParams& dp, const MdParams& md, int64_t N, const double* pos,
                        double* vel, const void* force, bool f64, unsigned long long* step, double* kpart,
                        double* stats, unsigned* done);
int md_blocks(int64_t N);

// Per-k coefficients of the current batch (one record per sampled k).
struct KCoef {
    int nx, ny, nz, ok;
    double kx, ky, kz, c;               // c = -coef / k^2
    double E, Ore, Oim;                 // E = Y_even, O = conj(Y_odd)  (Sec. 3.4)
    double dE_t, dE_b, dOre_t, dOim_t, dOre_b, dOim_b;
};

// Force-kernel record per k, FP32 mode: integer indices for the exact phase, the
// wave vector and the pre-scaled A' = c A, B' = c B.  48 bytes, three 16-byte loads.
struct __align__(16) KRec32 {
    int nx, ny, nz, pad0;
    float kx, ky, kz, pad1;
    float Ar, Ai, Br, Bi;
};

// Force-kernel records of the FP32 path, two wave vectors k0 = 2p, k1 = 2p + 1 per record
// (component x: k0, y: k1) so the force kernel runs its float32 arithmetic on both with
// paired instructions.  A' = c A, B' = c B and their negations; the first 80 bytes are
// all that the force without potential reads.  An odd P leaves the k1 half of the last
// record zero (the buffer is cleared at set-up and that half is never written).
struct __align__(16) KPair32 {
    int2 nx, ny;
    int2 nz;
    float2 kz;
    float2 kx, ky;
    float2 nAr, Ai;  // -A'_r, A'_i
    float2 nBr, Bi;  // -B'_r, B'_i
    float2 Ar, Br;   // A'_r, B'_r (potential only)
};
static_assert(sizeof(KPair32) == 96, "KPair32 is six 16-byte loads");
static_assert(offsetof(KPair32, Ar) == 80, "the potential-only fields come last");

// FP64 mode record.
struct __align__(16) KRec64 {
    long long nx, ny, nz, pad0;
    double kx, ky, kz, pad1;
    double Ar, Ai, Br, Bi;
};

// Packed particle, FP64 mode: 64-bit fixed-point fractional coordinates and q.
struct __align__(16) Part64 {
    unsigned long long ux, uy, uz;
    double q;
};

// Scalars written by the finalize step (device, float64).
enum ScalarSlot {
    SC_UK = 0, SC_USELF = 1, SC_UIBC = 2, SC_UREAL = 3,
    SC_Q = 4, SC_Q2 = 5, SC_MU = 6, SC_QABS = 7,
    SC_FIBC = 8,      // F_IBC,z = q_i * SC_FIBC
    SC_DQ_IBC_Z = 9,  // dU_IBC/dq_i = z_i * SC_DQ_IBC_Z + SC_DQ_IBC_C
    SC_DQ_IBC_C = 10,
    SC_DG_T = 11, SC_DG_B = 12,
    SC_ZMIN = 13, SC_ZMAX = 14,
    SC_UK_ACC = 15,  // running sum of U_k over the chunks of a lattice sum
    SC_COUNT = 16
};

// Device status words: k-sampler exhaustion, bounded-wait timeouts, and cell-list work
// limits (a cell too crowded to order, a charge with too many neighbour candidates, or a
// non-finite MD coordinate), each reported by rbe2d_sync_status.
enum StatusSlot { ST_SAMPLER = 0, ST_TIMEOUT = 1, ST_CELL = 2, ST_MD = 3, ST_COUNT = 4 };

// Work limits that keep the cell-list kernels bounded whatever the configuration.
constexpr int kMaxOrderedCell = 4096;      // larger cells keep their scatter order
constexpr int kMaxCandidates = 1 << 16;    // neighbour candidates examined per charge

// Pack partial-sum layout per block: Q, Q2, mu, Qabs, zmin, zmax.
constexpr int PACK_STRIDE = 8;

// Sampler tables on the device: per dimension the normalised cumulative table and a
// guide table (guide[g] = first index whose value exceeds g / len).
struct SamplerTables {
    const double* cdf[3];
    const int* guide[3];
    const double* w[3];  // the 1-D factors themselves (Metropolis variant)
    int len[3];
    int hw[3];           // Metropolis proposal half-widths
    const double* eo;    // image-series sums per kz (9 float64 per row), rows kz = -eo_half .. eo_half
    int eo_half;
};

// ---------------------------------------------------------------- launchers
// Process-wide count of kernel launches made by this library (rbe2d_kernel_launches);
// every launcher adds the number of kernels it enqueued.
void note_launches(int n);

// All launchers enqueue on `st` and return cudaGetLastError().
// step_dev != NULL: the step number is read on the device (graph replays advance it).
// tb.eo / tb.eo_half: the per-kz image-series table of the sampler's box (set-up).
cudaError_t launch_sample(cudaStream_t st, const DevParams& dp, const SamplerTables& tb, uint64_t seed,
                          uint64_t step, const unsigned long long* step_dev, KCoef* kc, int32_t* kidx_out,
                          int* status);
cudaError_t launch_set_k(cudaStream_t st, const DevParams& dp, const int32_t* kidx, KCoef* kc,
                         int* status);
// Per-kz table of the nine image-series sums for kz = -half .. half (set-up, once).
cudaError_t launch_eo_table(cudaStream_t st, const DevParams& dp, int half, double* eo);
// Metropolis variant: advance the P chains in `state` by `sweeps` updates of step `step`
// and make their states the batch.
cudaError_t launch_metropolis(cudaStream_t st, const DevParams& dp, const SamplerTables& tb, uint64_t seed,
                              uint64_t step, int sweeps, int32_t* state, KCoef* kc, int32_t* kidx_out,
                              unsigned long long* accepted);
// Entries [t0, t0 + P) of the half lattice {0 < (nz, ny, nx) lexicographically, |n_d| <= nm[d]}
// with weights 2 exp(-k^2/4alpha^2); slots past n_half get weight 0.
cudaError_t launch_lattice_k(cudaStream_t st, const DevParams& dp, const int nm[3], int64_t t0, int64_t n_half,
                             KCoef* kc);
// scal[SC_UK_ACC] = (first ? 0 : scal[SC_UK_ACC]) + scal[SC_UK]; last: scal[SC_UK] = scal[SC_UK_ACC].
cudaError_t launch_accum_uk(cudaStream_t st, double* scal, int first, int last);
// Internal flag of launch_force: leave the self term out of phi (all but the first chunk
// of a lattice sum).
constexpr int kForceNoSelf = 1 << 30;
cudaError_t launch_pack(cudaStream_t st, const DevParams& dp, int64_t N, const void* pos,
                        const void* q, bool in_f32, bool fp64, void* part, double* pack_part,
                        int pack_blocks);
int pack_blocks_for(int64_t N);
// FP64 mode: structure factor of packed particles (pack_kernel runs first).
cudaError_t launch_sf64(cudaStream_t st, const DevParams& dp, int64_t N, const void* part, bool want_sigma,
                        const KCoef* kc, double* sf_part, int nblk, int kthreads, int kchunks);
// FP32-mixed mode: structure factor with packing fused (writes part and pack_part).
// host_inputs: pos and q are pinned host memory read in place (the first tile is then
// staged in pieces; the results are the same bits either way).
cudaError_t launch_sf32(cudaStream_t st, const DevParams& dp, int64_t N, const void* pos, const void* q,
                        bool in_f32, bool want_sigma, const KCoef* kc, double* sf_part, int nblk, int kthreads,
                        int kchunks, void* part, double* pack_part, int npoly, bool host_inputs, int shape);
// The variants of the FP32-mixed structure factor that skip wave-vector groups holding
// no k below P (launch_sf32 chooses them; sf32_live.cu).
void launch_sf32_live(cudaStream_t st, dim3 grid, int kthreads, int npoly, int shape, bool in_f32, bool sig,
                      const DevParams& dp, const void* pos, const void* q, int64_t N, const KCoef* kc,
                      double* sf_part, int nblk, uint4* po, double* pack_part);
// Fold (one warp per k) with the finalize step run by the last CTA; `done` must be zero
// before the launch and is zero again after it.
cudaError_t launch_fold(cudaStream_t st, const DevParams& dp, const double* sf_part, int nblk,
                        const KCoef* kc, bool fp64, double* rs, double* kterm, void* krec,
                        const double* pack_part, int pack_blocks, double* pack2, double* scal, unsigned* done);
// The grid is one wave of resident CTAs of the chosen shape (fshape, FP32 mode), or fewer
// when N has fewer rounds.  fpoly and fshape are the choice for the variant that runs:
// the potential variant's (kPot* shapes) when flags has RBE2D_POTENTIAL and phi is set.
cudaError_t launch_force(cudaStream_t st, const DevParams& dp, int64_t N, const void* part,
                         bool fp64, const void* krec, const double* scal, int flags, void* force,
                         void* phi, double fscale, double pscale, const struct Shapes& sh, unsigned* counters,
                         int fpoly, int fshape);
cudaError_t launch_copy_energy(cudaStream_t st, const double* scal, double* energy_out);
cudaError_t launch_dgamma(cudaStream_t st, const double* scal, double g, double* dgamma);
cudaError_t launch_inject_totals(cudaStream_t st, int P, const double* rho, const double* sums, double* sf_part,
                                double* pack_part);
cudaError_t launch_copy_sums(cudaStream_t st, const double* scal, double* out);

// Real-space cell grid: cells of at least r_c in x, y (periodic) and in z over
// [z0, z0 + ncz hz] = [-r_c, H + r_c]; neighbours within mx, my cells (and one in z);
// images up to level lmax can lie within r_c of the slab.
struct CellGrid {
    int ncx, ncy, ncz, ncell, mx, my, lmax;
    double hx, hy, hz, z0;
    double inv_hx, inv_hy, inv_hz;
};

struct RealBuffers {
    int* count;         // [ncell]
    int* start;         // [ncell + 1]
    int* fill;          // [ncell]
    int* tile_sum;      // [ceil(ncell / 1024)] per-tile source counts of the scan
    void* src;          // [nsrc_max] float4 / double4 (corner-relative x, y, z; q g)
    void* src_sorted;   // the same, in key order within each cell
    long long* key;     // [nsrc_max] particle index * 256 + image slot
    long long* key_sorted;
    double* epart;      // [ncell] energy partial sums
    int64_t nsrc_max;
};

// Sorted cell list of the sources (real charges and their images within dp.r_c of the
// slab) on grid g.  gate != NULL: every kernel returns at once unless *gate != 0.
// count_real != NULL: also the real charges per cell and their exclusive scan real_start
// (ncell + 1 entries; tile_sum2: scan tiles).  max_blocks > 0 caps the grids of the
// grid-stride kernels (a gated launch that returns at once then costs one short launch).
cudaError_t launch_cells(cudaStream_t st, const DevParams& dp, const CellGrid& g, const RealBuffers& rb, int64_t N,
                         const void* pos, const void* q, bool in_f32, bool fp64, int* status, const int* gate,
                         int* count_real, int* real_start, int* tile_sum2, int max_blocks = 0);
cudaError_t launch_real(cudaStream_t st, const DevParams& dp, const CellGrid& g, const RealBuffers& rb, int64_t N,
                        const void* pos, const void* q, bool in_f32, bool fp64, void* force, void* phi, int pot,
                        int energy, double* scal, unsigned* done, int* status);

// Real-space pair lists of the MD loop (FP32-mixed mode; pairlist_kernels.cu).  Entry
// encoding: particle * kNlMaxSlots + image slot.
constexpr int kNlMaxSlots = 64;
struct PairLists {
    double skin;          // pairs within r_c + skin are listed
    CellGrid g;           // cells of at least r_c + skin; g.lmax: image levels within r_c + skin
    int cap;              // entries per charge
    int64_t n_slots;      // list columns (n_max): entry e of slot t at nl[e * n_slots + t]
    int* nl;              // [cap][n_slots]: source slot * 64 + image slot
    int* cnt;             // [n_slots] entries of each slot
    int* tgt;             // [n_slots] particle of each slot (charges in cell order)
    uint4* rec;           // [n_max] this step's fixed-point records {ux, uy, A, q}
    uint4* ref;           // [n_max] the records at the last build
    uint4* srec;          // [n_slots] this step's records in slot (cell) order: srec[t] = rec[tgt[t]]
    int* inv;             // [n_max] slot of each particle (inverse of tgt)
    int* count_real;      // [ncell] charges per cell of the list grid
    int* real_start;      // [ncell + 1] their exclusive scan: the first slot of each cell
    int* tile_sum2;       // scan tiles of count_real
    int* flag;            // [0]: rebuild before the next evaluation (set at set-up and by the prep kernel)
    int build_blocks;     // grid of the build kernel (it loops over the cells)
    unsigned long long* builds;  // number of builds so far
};
// One real-space (and WCA) force evaluation of the MD loop through the lists, rebuilt first
// on the device when the flag is set: pos, q float64 device arrays; the float32 force is
// added to force.
cudaError_t launch_real_lists(cudaStream_t st, const DevParams& dp, const PairLists& L, const RealBuffers& rb,
                              int64_t N, const double* pos, const double* q, float* force, int* status);

// ---------------------------------------------------------------- batched systems
constexpr int kBatchKR = 4;  // wave vectors per thread in batched structure-factor items (P <= 512)

struct BatchSys {
    DevParams dp;
    long long off, N;          // particle range [off, off + N) in the concatenated arrays
    int nsf, nf;               // structure-factor and force items of this system
    int sf_base, f_base;       // first item of each kind (force items counted from 0)
    long long part_base;       // offset of this system's [P][nsf][4] partial sums
    int tab_off[3], tab_len[3];  // sampler tables inside the concatenated arrays
    unsigned long long seed;
    long long eo_off;          // this system's per-kz image-series table (float64 offset)
    int eo_half;               // its rows are kz = -eo_half .. eo_half
};

struct BatchArgs {
    const BatchSys* sys;
    int n_sys, P_max;
    const int* item_sys;       // system of every item (structure-factor items first)
    int n_sf_items, n_f_items, sf_chunk, f_chunk;
    const double* pos;
    const double* q;
    float* force;
    int ibc;
    const KCoef* kc;
    const double* eo;          // the systems' per-kz image-series tables (9 float64 per row)
    KPair32* krec;             // [system][KP] force records, two wave vectors each
    int KP;                    // records per system: (P_max + 1) / 2
    uint4* part;               // [sum N] fixed-point particle records {ux, uy, uz, q}
    double* partial;
    double* pack;              // [structure-factor item][4]: Q, Q2, mu
    double* scal;              // [system][4]: U_k, U_self, U_IBC, F_IBC factor
    int* sf_done;
    int* ready;
    int* head;
    unsigned* exit_count;
    int* status;
    unsigned long long wait_ns;  // bound of a force item's wait for its system's fold
    int withhold;              // system whose ready flag is not published (timeout tests), or -1
};

// variant 0: registers as needed; 1: capped for 8 resident CTAs per SM (P_max <= 256).
cudaError_t launch_batch(cudaStream_t st, const BatchArgs& a, int grid, int variant);
cudaError_t launch_batch_sample(cudaStream_t st, const BatchArgs& a, const double* cdf, const int* guide,
                                uint64_t step);
cudaError_t batch_occupancy(int P_max, int variant, int* per_sm);

// Launch shapes of the FP32-mixed kernels that the autotuner chooses from.
// Structure factor: wave vectors per thread (KR), particles per shared-memory tile and the
// resident CTAs per SM the register budget is cut for.  Shapes 1 and 2 exist for
// float64 inputs in device memory (the other input kinds run shape 0).
// FMA-pipe sin/cos share levels of the tuner (0, 1, 2, 4 angles in each group of 8).
constexpr int kPolyLevels = 4;
constexpr int kSfShapes = 3;
constexpr int kSfKR[kSfShapes] = {4, 4, 2};
constexpr int kSfTile[kSfShapes] = {224, 448, 224};
constexpr int kSfMinBlocks[kSfShapes] = {8, 5, 8};
// Force: threads per CTA, particles per thread, the resident CTAs per SM the register
// budget is cut for (0: no cut) and the threads sharing one particle's k-sum (a round is
// threads x particles / split).
constexpr int kForceShapes = 7;
constexpr int kForceThreads[kForceShapes] = {256, 128, 256, 512, 256, 256, 256};
constexpr int kForceR[kForceShapes] = {2, 2, 1, 2, 2, 1, 1};
constexpr int kForceMinBlocks[kForceShapes] = {0, 0, 0, 0, 5, 0, 0};
constexpr int kForceSplit[kForceShapes] = {1, 1, 1, 1, 1, 2, 4};  // threads per particle (k-split)
// The potential variant of the force kernel (RBE2D_POTENTIAL: dU/dq beside the force;
// the adjoint) carries four more sums and takes its own shapes, chosen by
// rbe2d_autotune_potential: 256 x 2 cut to 64 registers (4 CTAs per SM) with the k-sum
// in 1, 2 or 4 threads, and 256 x 1 cut to 40 registers (6 CTAs per SM).
constexpr int kPotShapes = 4;
constexpr int kPotThreads[kPotShapes] = {256, 256, 256, 256};
constexpr int kPotR[kPotShapes] = {2, 2, 2, 1};
constexpr int kPotMinBlocks[kPotShapes] = {4, 4, 4, 6};
constexpr int kPotSplit[kPotShapes] = {1, 2, 4, 1};

// Occupancy-derived launch shapes (queried once at init).
struct Shapes {
    int sms;
    int sf_threads32[kSfShapes], sf_threads64;  // threads per CTA of the structure-factor kernels
    int sf_occ32[kSfShapes], sf_occ64;          // resident CTAs per SM
    int force_threads;
    int force_occ32[kForceShapes], force_occ64;
    int pot_occ32[kPotShapes];  // the potential variant's shapes
};
cudaError_t query_shapes(int device, int P_pad, Shapes* sh);
// Resident CTAs per SM of the FP32 and FP64 force kernels for a batch of P_pad k.
cudaError_t force_occupancy(int P_pad, int* occ32, int* occ64);
cudaError_t pot_occupancy(int P_pad, int* occ32);  // the potential variant's shapes

}  // namespace rbe2d
