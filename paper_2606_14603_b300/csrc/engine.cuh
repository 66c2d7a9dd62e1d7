// engine.cuh — device-side data layout and helpers of the step engine.
//
// Layout in HBM (one arena per batch, 256-byte aligned sub-buffers):
//   pm[2][C]     int4 agent record, double-buffered: the position packed as
//                x | y << 21 | z << 42 in the first two words (positions in
//                [0, 2^21) units), the meta word, the agent id (per simulation)
//   apar[2][C]   u32 partner id         (valid for carriers only)
//   rk[C]        u32 rank within the new cell, from the move pass (the
//                scatter finds the cell again from the moved record)
//   acc[C]       u64 proposal slot, min of (dist^2 << 32 | proposer id)
//   props[C]     (proposer, target) sorted indices of this step's proposals
//   pflag[C]     1 if the sorted agent is a free proposer (written by the scatter)
//   xpm/xrk      released partners appended by the move pass (C/2 + 1): record, rank
//   bseg[S][Q]   births of the step, one segment of Q per simulation slot:
//                (parent's slot in the moved buffer, parent id)
//   bofs[S+1]    births placed before each simulation this step (prefix)
//   bsrt[S][Q]   parent ids of a long births segment, sorted tile by tile
//                (kBirthTile entries each), for the ranking by binary search
//   btofs[S+1]   sorted tiles before each simulation this step (prefix)
//   cnt[K], start[K+1]  per-cell histogram and its exclusive scan
//   tcnt[T]      agents per cell tile (8192 cells), counted by the move pass,
//                one counter per 128-byte line (kTileStride words apart) so
//                that the atomics of different tiles meet in different L2 lines
//   tsum[T+1]    exclusive tile prefixes (grids of more than kDirectTiles tiles)
//   sims[S], models[S], obs (counts/digests), live[2][S][512], ctl
//
// Step-local counters (released partners, proposals, births) are indexed by
// the parity of the global step counter `epoch`: a step with epoch E uses
// parity E & 1, and the bookkeeping block of k_scan (which advances epoch
// to E + 1) clears the counters of the other parity for the next step, so
// no kernel ever resets a counter another kernel of the same step reads.
//
// meta word: bits 0-5 species, 6-7 compartment, 8 carrier, 9 carrier is
// reactant a, 10 dead, 11 absorbed (became hidden this step), 12-19 reaction
// of the complex, 20-30 simulation slot, 31 the species proposes (kept in
// step with every change of species).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace abm {

constexpr int kMaxSpecies = 64;
constexpr int kMaxReactions = 255;
constexpr int kMaxComp = 4;
constexpr int kMaxSims = 2048;
constexpr uint32_t kDefaultBirths = 8192;   // default births per step of one simulation
constexpr uint32_t kBirthTile = 2048;       // births segments longer than this are ranked through sorted tiles
constexpr uint32_t kSortBlocks = 16;        // blocks of k_scan that sort those tiles
constexpr int kScanTile = 8192;           // cells per scan tile (256 threads x 32)
constexpr int kTileStride = 32;           // words between two tile counters
constexpr uint32_t kDirectTiles = 8192;   // up to this many tiles, each scan block adds up its own prefix
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kMonTrace = 1024;      // evaluations kept per threshold monitor
constexpr uint64_t kEmpty = 0xFFFFFFFFFFFFFFFFull;

constexpr uint32_t M_SP = 0x3Fu;
constexpr uint32_t M_COMP_SHIFT = 6, M_COMP = 0xC0u;
constexpr uint32_t M_BOUND = 1u << 8;
constexpr uint32_t M_ROLE_A = 1u << 9;
constexpr uint32_t M_DEAD = 1u << 10;
constexpr uint32_t M_ABSORBED = 1u << 11;
constexpr uint32_t M_RXN_SHIFT = 12, M_RXN = 0xFFu << 12;
constexpr uint32_t M_SIM_SHIFT = 20, M_SIM_MASK = 0x7FFu;
constexpr uint32_t M_PROP = 1u << 31;       // free agent of a species that proposes

// device error codes (ctl.err); mapped to abm_status on the host
enum : uint32_t {
    ERR_NONE = 0,
    ERR_CAPACITY_AGENTS = 1,
    ERR_CAPACITY_EXTRAS = 2,
    ERR_CAPACITY_BIRTHS = 3,
    ERR_PLACEMENT = 5,
    ERR_ID_SPACE = 6,
    ERR_CAPACITY_DUMP = 7,
};
// per-simulation error codes (SimDev.err): the simulation stops, the batch goes on
enum : uint32_t {
    SIM_ERR_BIRTHS = 1,      // births of one step beyond the simulation's limit
};

struct SpeciesDev {          // 48 bytes
    uint64_t thr_uni, thr_emit, thr_cross;
    uint64_t partner_mask;   // bit b: a reaction (this species, b) exists
    uint32_t M;              // Gaussian multiplier, 0 = immobile
    int16_t uni_to, emit;    // -1 = death / none
    uint16_t has_event;      // thr_uni or thr_emit nonzero
    uint16_t init_comp;      // compartment of the initial agents
    int32_t rmax;            // largest contact radius over the reactions it proposes
};

struct ReactionDev {         // 32 bytes
    uint64_t thr_bind, thr_rel;
    uint32_t R2;
    int32_t R;
    int16_t prod_a, prod_b;
    uint8_t kind, carrier_a, a, b;
};

struct ModelDev {
    SpeciesDev sp[kMaxSpecies];
    ReactionDev rx[kMaxReactions + 1];
    uint8_t rx_of[kMaxSpecies][kMaxSpecies];  // 0xFF = none
    uint32_t n_sp, n_rx, n_comp, n_counts;
};

struct SimDev {              // per simulation slot
    uint32_t active;         // 1 while stepping
    uint32_t model;
    uint32_t key0, key1;     // Philox key = seed
    uint32_t step;           // local step t
    uint32_t next_id;
    int32_t ext;             // positions in [0, ext]
    int32_t root_sphere;
    int64_t root_r2;
    int32_t c0[3];
    int32_t n_comp;
    int32_t cc[kMaxComp][3]; // child centres (index 1..)
    int64_t cr2[kMaxComp];   // child radius^2
    uint32_t shift;          // cell edge 2^shift
    uint32_t g;              // cells per axis
    uint32_t cell_off;       // first global cell
    uint32_t n_counts;       // counts vector length
    uint32_t counts_off;     // offset into the counts buffer
    uint32_t max_step;       // the sim is frozen (kept, not advanced) once step reaches this
    // step-local words (written on the device each step)
    uint32_t tau;            // step index of the step in flight (read by the proposal search)
    uint32_t adv;            // 1: the step in flight advances this simulation
    uint32_t nbc[2];         // births reserved by the move pass, by step parity
    uint32_t nb;             // births placed by the step in flight
    uint32_t nid0;           // id of the step's first child (next_id before the step's births)
    uint32_t err;            // per-simulation error (SIM_ERR_*), sticky; the simulation is frozen
    uint32_t err_info;
    uint32_t nbt;            // sorted tiles of this step's births (0: ranked by direct comparison)
    uint32_t pad_sim;
};

// Threshold monitor of one simulation slot (Sec. 2: designated species
// followed against a threshold inside a time window).  value(t) = sum over
// the counts vector of weight * count at the state after t completed steps.
struct MonDev {
    uint32_t active;
    uint32_t begin, end, period;   // evaluated at t in [begin, end), (t - begin) % period == 0
    int64_t threshold;
    uint32_t above;          // 1: passes when value > threshold; 0: when value < threshold
    uint32_t n_eval, n_passed;
    uint32_t last_step;      // step of the last evaluation
    uint32_t first_pass;     // first evaluated step that passed, kNone = none
    int32_t state;           // outcome of the last evaluation, -1 = none yet
    int64_t value;           // value at the last evaluation
};

struct Ctl {
    uint32_t n_buf[2];       // agents in buffer 0 / 1
    uint32_t cur;            // buffer holding the state between steps (flipped by k_scan's bookkeeping)
    uint32_t n_sorted;       // agents placed by this step's scatter
    uint32_t n_cells;        // cells in use
    uint32_t epoch;          // global step counter (1 + steps run)
    uint32_t err;
    uint32_t err_info;
    uint32_t n_sims;         // sim slots in use (upper bound of the table)
    uint32_t dump_n;
    uint32_t n_monitors;     // simulations with an active threshold monitor
    uint32_t n_extra[2];     // released partners, by step parity
    uint32_t n_props[2];     // proposals (list in props), by step parity
    uint32_t nb_total;       // births placed by the step in flight
    uint32_t live_counts;    // 1: each step leaves the counts of its result in live[epoch & 1]
    uint32_t n_compact;      // agents kept by a compaction (between steps)
    uint32_t sim_errs;       // simulations that raised a per-simulation error
    uint32_t move_parity;    // epoch & 1 of the step in flight, written by its move pass
    uint32_t pad[2];
};

struct Buffers {
    int4* pm[2];             // packed records (pack_rec)
    uint32_t* apar[2];
    uint32_t* rk;            // per agent: rank within its new cell (kNone: not placed)
    uint64_t* acc;
    uint2* props;
    uint8_t* pflag;
    int4* xpm;
    uint32_t* xrk;
    uint2* bseg;             // [max sims][bquota] births: (parent slot, parent id)
    uint32_t* bofs;          // [max sims + 1] births before each simulation this step
    uint32_t* bsrt;          // [max sims][bquota] parent ids of long segments, sorted per tile
    uint32_t* btofs;         // [max sims + 1] sorted births tiles before each simulation
    uint32_t* cnt;
    uint32_t* start;
    uint32_t* tcnt;
    uint32_t* tsum;
    SimDev* sims;
    ModelDev* models;
    uint64_t* counts;
    uint64_t* live;          // [2][max sims][512]: counts of a step's result, by step parity
    uint64_t* digests;
    MonDev* mons;            // [max_sims]
    int32_t* mon_w;          // [max_sims][512] weights over the counts vector
    uint64_t* mon_acc;       // [max_sims] running sums (two's complement)
    int64_t* mon_trace;      // [max_sims][kMonTrace] ring of evaluated values
    const int16_t* ztab;
    Ctl* ctl;
    uint64_t cap_agents;
    uint64_t cap_extras;
    uint64_t cap_cells;
    uint32_t bquota;         // births per step of one simulation (segment length)
    uint32_t n_tiles_max;
    uint32_t propose_chunk;  // sorted agents per proposal-search block round (multiple of 256)
    uint32_t live_stride;    // entries of one live-counts buffer (max sims x 512)
    uint32_t max_sims;       // simulation slots
};

// Packed agent record: the position x | y << 21 | z << 42 in words 0-1,
// the meta word, the id.  Positions lie in [0, kPosLimit).
constexpr int32_t kPosLimit = 1 << 21;
__host__ __device__ __forceinline__ int4 pack_rec(int32_t x, int32_t y, int32_t z, uint32_t meta, uint32_t id) {
    return make_int4((int)((uint32_t)x | (uint32_t)y << 21), (int)((uint32_t)y >> 11 | (uint32_t)z << 10),
                     (int)meta, (int)id);
}
// The unpacked view {x, y, z, meta} of a packed record (its id is r.w).
__host__ __device__ __forceinline__ int4 unpack_rec(int4 r) {
    const uint32_t a = (uint32_t)r.x, b = (uint32_t)r.y;
    return make_int4((int)(a & 0x1FFFFFu), (int)(a >> 21 | (b & 0x3FFu) << 11), (int)(b >> 10), r.z);
}
// A record from its unpacked view p ({x, y, z, meta}) and id.
__host__ __device__ __forceinline__ int4 repack(const int4& p, uint32_t id) {
    return pack_rec(p.x, p.y, p.z, (uint32_t)p.w, id);
}

// The live-counts buffer a step with this epoch fills.
__device__ __forceinline__ uint64_t* live_buffer(const Buffers& B, uint32_t epoch) {
    return B.live + (size_t)(epoch & 1u) * B.live_stride;
}

// ------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64 multiplies with Weyl-sequence key bumps between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)c.x * 0xD2511F53u;  // one 32x32->64 product each
        const uint64_t p1 = (uint64_t)c.z * 0xCD9E8D57u;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    }
    return c;
}

// Gaussian step: sign-magnitude, rounded half up, so d(-Z) = -d(Z) exactly.
__device__ __forceinline__ int32_t gauss_step(int32_t z, uint32_t M) {
    const uint32_t mag = (uint32_t)(z < 0 ? -z : z);
    const uint32_t d = (uint32_t)(((uint64_t)mag * M + 0x80000000ull) >> 32);
    return z < 0 ? -(int32_t)d : (int32_t)d;
}

// Fold about the half-integer walls -1/2 and ext+1/2 (counting-measure
// preserving reflection).  |v - x| <= ext guarantees one fold suffices.
__device__ __forceinline__ int32_t fold(int32_t v, int32_t ext) {
    if (v < 0) return -v - 1;
    if (v > ext) return 2 * ext + 1 - v;
    return v;
}

__device__ __forceinline__ int64_t d2c(int32_t x, int32_t y, int32_t z, const int32_t* c) {
    const int64_t dx = x - c[0], dy = y - c[1], dz = z - c[2];
    return dx * dx + dy * dy + dz * dz;
}

// Compartment holding a point; -1 outside a spherical root.
__device__ __forceinline__ int locate(const SimDev& S, int32_t x, int32_t y, int32_t z) {
    if (S.root_sphere && d2c(x, y, z, S.c0) > S.root_r2) return -1;
    for (int k = 1; k < S.n_comp; k++)
        if (d2c(x, y, z, S.cc[k]) <= S.cr2[k]) return k;
    return 0;
}

__device__ __forceinline__ uint32_t cell_of(const SimDev& S, int32_t x, int32_t y, int32_t z) {
    const uint32_t g = S.g;
    return S.cell_off + ((uint32_t)(z >> S.shift) * g + (uint32_t)(y >> S.shift)) * g +
           (uint32_t)(x >> S.shift);
}

// MurmurHash3 64-bit finaliser (Appleby), for the order-independent digest.
__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

__device__ __forceinline__ uint64_t record_hash(uint32_t id, uint32_t sp, uint32_t comp, uint32_t flags,
                                                uint32_t rxn, int32_t x, int32_t y, int32_t z,
                                                uint32_t partner) {
    uint64_t h = fmix64((uint64_t)id | (uint64_t)sp << 32 | (uint64_t)comp << 40 |
                        (uint64_t)flags << 48 | (uint64_t)rxn << 56);
    h = fmix64(h ^ ((uint64_t)(uint32_t)x | (uint64_t)(uint32_t)y << 32));
    h = fmix64(h ^ ((uint64_t)(uint32_t)z | (uint64_t)partner << 32));
    return h;
}

__host__ __device__ __forceinline__ uint32_t sim_of(uint32_t meta) { return (meta >> M_SIM_SHIFT) & M_SIM_MASK; }

// meta with species sp, the proposer bit following the species
__device__ __forceinline__ uint32_t with_species(uint32_t meta, uint32_t sp, const ModelDev& Mo) {
    meta = (meta & ~(M_SP | M_PROP)) | sp;
    return Mo.sp[sp].partner_mask ? meta | M_PROP : meta;
}

__device__ __forceinline__ void raise_error(Ctl* ctl, uint32_t code, uint32_t info) {
    if (atomicCAS(&ctl->err, 0u, code) == 0u) ctl->err_info = info;
}

// Index of a live record in the counts vector: free agents by (species,
// compartment), bound carriers by reaction (one entry per bound pair).
__device__ __forceinline__ uint32_t count_slot(uint32_t meta, const ModelDev& Mo) {
    if (meta & M_BOUND) return Mo.n_sp * Mo.n_comp + ((meta & M_RXN) >> M_RXN_SHIFT);
    return (meta & M_SP) * Mo.n_comp + ((meta & M_COMP) >> M_COMP_SHIFT);
}

// Whether a monitor evaluates the state after t completed steps (each such
// state at most once, whether in a step or at a read between steps).
__device__ __forceinline__ bool mon_due(const MonDev& M, uint32_t t) {
    return M.active && t >= M.begin && t < M.end && (t - M.begin) % M.period == 0 &&
           (M.n_eval == 0 || t > M.last_step);
}

// ------------------------------------------------------------------------
// Host-side launch wrappers (kernels.cu).
struct Launch {
    int blocks_agents;       // grid of the between-step per-agent kernels (grid-stride, 256 threads)
    int blocks_move;         // grid of k_move: the blocks of threads_move that fit at once
    int blocks_move_live;    // the same for its live-counting variant (more registers, maybe fewer blocks)
    int blocks_scatter;      // grid of k_scatter (same block size): the blocks that fit at once
    int threads_move;        // block size of k_move and k_scatter: 128, 256 or 512
    bool dense_move;         // k_move in 48 registers (five 256-thread blocks per SM): batches above 2M agents
    int threads;             // 256
    int blocks_scan;
    int blocks_accept;       // CTAs of the acceptance kernel (walks the proposal list)
    int blocks_propose;      // CTAs of the proposal search, one chunk of sorted agents each
    bool prefix_kernel;      // more than kDirectTiles tiles: tile prefixes by k_tile_prefix
};

// CTAs of k_move with `threads` threads that fit on one SM at once (its
// registers decide; dense: the 48-register variant; live: the variant that
// keeps live counts); valid block sizes are 128, 256 and 512.
int move_blocks_per_sm(int threads, bool dense = false, bool live = false);
int scatter_blocks_per_sm(int threads);
bool valid_move_threads(int threads);
size_t propose_smem(const Buffers& B);

cudaError_t prepare_kernels();
// live: the move pass variant that also keeps live counts (ctl.live_counts on)
cudaError_t launch_step(const Buffers& B, const Launch& L, cudaStream_t s, bool live = false);

cudaError_t launch_init(const Buffers& B, const Launch& L, cudaStream_t s, uint32_t sim,
                        uint32_t base, uint32_t n0, const uint32_t* d_species_end, uint32_t n_sp);
cudaError_t launch_observe(const Buffers& B, const Launch& L, cudaStream_t s, int32_t only_sim, int want_digest);
// The step with a CUDA event before and after each of its kernels (ev[0..6]).
constexpr int kStepKernels = 6;
cudaError_t launch_step_timed(const Buffers& B, const Launch& L, cudaStream_t s, cudaEvent_t* ev,
                              bool live = false);
// Between steps: drop the agents of retired simulations (counter: ctl.n_sorted).
cudaError_t launch_compact(const Buffers& B, const Launch& L, cudaStream_t s);
cudaError_t launch_dump(const Buffers& B, const Launch& L, cudaStream_t s, int32_t sim, void* d_out,
                        uint32_t cap);
// Threshold monitor of one simulation at the current state (between steps):
// adds up its value if that state is due and not yet evaluated, then evaluates.
cudaError_t launch_monitor(const Buffers& B, const Launch& L, cudaStream_t s, int32_t sim);
// Counts vector (n <= 512 words) and control words into a pinned host slot of
// 512 + sizeof(Ctl) / 8 words (device-visible under unified addressing).
cudaError_t launch_readout(const uint64_t* src, uint32_t n, const Ctl* ctl, uint64_t* dst, cudaStream_t s);
cudaError_t launch_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n,
                                cudaStream_t s);

}  // namespace abm
