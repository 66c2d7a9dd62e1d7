// kernels.cu — the per-step CUDA kernels (sm_103a) of the molecule-agent engine.
//
// One step (paper Sec. 2: diffusion, proximity binding, product release,
// expression, degradation, compartment migration) is five launches over the
// whole batch of simulations (six on grids of more than 8192 scan tiles),
// all reading their sizes from the device control block so that a captured
// CUDA graph replays them unchanged:
//
//   k_move      P1 events + P2 Brownian move + cell key + histogram rank
//               (and agents per tile of 8192 cells); births are reserved in
//               their simulation's segment
//   k_tile_prefix  prefixes of the per-tile agent counts (grids of more
//               than 8192 tiles only)
//   k_scan      exclusive scan of the cell histogram, tile prefixes included;
//               one extra block does the step's bookkeeping meanwhile (births
//               per simulation, monitors, step counters, buffer flip), and
//               16 more sort the tiles of long births segments by parent id
//   k_scatter   reorder every live agent by cell into the other buffer
//   k_propose   neighbour query over the cells a contact radius can reach,
//               nearest eligible partner, atomicMin on a packed key; births
//               ranked by parent id (directly, or by binary search over the
//               sorted tiles) and placed after the sorted agents
//   k_accept    final-edge rule and reaction application
//
// The engine never depends on storage order: every decision is a function
// of the set of (id, state) pairs, so atomics may run in any order.
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>

#include "engine.cuh"

namespace cg = cooperative_groups;

namespace abm {

namespace {

constexpr int kThreads = 256;

// Programmatic dependent launch: a step kernel may be launched while its
// predecessor finishes; it waits here until the predecessor's grid has
// completed and its writes are visible, and each block signals, when its
// work is done, that the successor may start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

// Warp-aggregated slot reservation: one atomicAdd per group of threads that
// reach this point together.
__device__ __forceinline__ uint32_t reserve(uint32_t* counter) {
    cg::coalesced_group g = cg::coalesced_threads();
    uint32_t base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, g.size());
    return g.shfl(base, 0) + g.thread_rank();
}

// P2 for one agent.  p.w carries the compartment bits, updated on crossing.
__device__ __forceinline__ void brownian_move(const SimDev& S, const SpeciesDev& sd,
                                              const int16_t* __restrict__ ztab, int4& p,
                                              uint32_t id, uint32_t t) {
    const uint32_t M = sd.M;
    if (M == 0) return;
    const uint4 m = philox(make_uint4(id, t, 0u, 0u), S.key0, S.key1);
    int32_t x = p.x + gauss_step(__ldg(&ztab[m.x >> 16]), M);
    int32_t y = p.y + gauss_step(__ldg(&ztab[m.y >> 16]), M);
    int32_t z = p.z + gauss_step(__ldg(&ztab[m.z >> 16]), M);
    if (!S.root_sphere) {
        x = fold(x, S.ext);
        y = fold(y, S.ext);
        z = fold(z, S.ext);
    }
    const int c = locate(S, x, y, z);
    if (c < 0) return;  // would leave the spherical cell: rejected
    const uint32_t comp = ((uint32_t)p.w & M_COMP) >> M_COMP_SHIFT;
    if ((uint32_t)c != comp) {
        if ((uint64_t)m.w >= sd.thr_cross) return;  // membrane: rejected
        p.w = (int)(((uint32_t)p.w & ~M_COMP) | ((uint32_t)c << M_COMP_SHIFT));
    }
    p.x = x;
    p.y = y;
    p.z = z;
}

// ------------------------------------------------------------------------
// k_move: P1 first-order events and P2 move for every agent of the current
// buffer, then the cell key and the agent's rank inside its cell (the value
// returned by the histogram atomic), which the scatter uses directly.
// Work of one agent of the move pass, in phases: events and the move draw,
// the step itself, then the results.
struct MoveState {
    int4 p;              // record, moved in place
    uint32_t id;
    uint32_t flags;      // 1 alive, 2 emit, 4 moves (M > 0)
    const SimDev* S;
    const ModelDev* Mo;
    uint32_t mw;         // crossing draw
    int32_t z[3];        // Gaussian table entries (loads in flight between phases)
    uint32_t key;
};

// Warp-aggregated add of each lane's monitor weight to its simulation's sum:
// the lanes of a warp nearly always belong to one simulation.
__device__ __forceinline__ void monitor_add(uint64_t* acc, uint32_t s, int32_t w) {
    const uint32_t mask = __activemask();
    const bool has = s != kNone && w != 0;
    const uint32_t live = __ballot_sync(mask, has);
    if (!live) return;
    const uint32_t s0 = __shfl_sync(mask, s, __ffs(live) - 1);
    const bool grp = has && s == s0;
    const uint32_t gmask = __ballot_sync(mask, grp);
    if (grp) {
        const int32_t sum = __reduce_add_sync(gmask, w);  // |w| <= 2^20: no overflow
        if ((threadIdx.x & 31u) == (uint32_t)(__ffs(gmask) - 1))
            atomicAdd((unsigned long long*)&acc[s0], (unsigned long long)(int64_t)sum);
    } else if (has) {
        atomicAdd((unsigned long long*)&acc[s], (unsigned long long)(int64_t)w);
    }
}

// A record's contribution to its simulation's monitor, if that monitor is
// due at the simulation's current step (only: a simulation, or kNone = any).
__device__ __forceinline__ void monitor_record(Buffers& B, uint32_t meta, uint32_t only) {
    uint32_t s = kNone;
    int32_t w = 0;
    if (!(meta & (M_DEAD | M_ABSORBED))) {
        const uint32_t sm = sim_of(meta);
        const SimDev& S = B.sims[sm];
        if ((only == kNone || sm == only) && S.active && mon_due(B.mons[sm], S.step)) {
            s = sm;
            w = B.mon_w[(size_t)sm * 512 + count_slot(meta, B.models[S.model])];
        }
    }
    monitor_add(B.mon_acc, s, w);
}

// Evaluates simulation s's monitor if the current state is due; run by one
// thread per simulation after every contribution has been added.
__device__ __forceinline__ void monitor_eval(Buffers& B, uint32_t s) {
    const SimDev& S = B.sims[s];
    if (!S.active) return;
    MonDev& M = B.mons[s];
    const uint32_t t = S.step;
    if (!mon_due(M, t)) return;
    const int64_t v = (int64_t)B.mon_acc[s];
    B.mon_acc[s] = 0;
    const bool passed = M.above ? v > M.threshold : v < M.threshold;
    B.mon_trace[(size_t)s * kMonTrace + M.n_eval % kMonTrace] = v;
    M.n_eval += 1;
    M.last_step = t;
    M.value = v;
    M.state = passed ? 1 : 0;
    if (passed) {
        M.n_passed += 1;
        if (M.first_pass == kNone) M.first_pass = t;
    }
}

// Phase 1: P1 events (a released partner is moved and placed right away:
// rare) and the move draw; issues the three table loads.  kLive: the step
// keeps live counts (the variant of the move pass launched while they are on).
template <bool kLive>
__device__ __forceinline__ void move_phase1(Buffers& B, Ctl* ctl, uint32_t cur, uint32_t parity, uint32_t i,
                                            MoveState& a) {
    uint32_t meta = (uint32_t)a.p.w;
    a.flags = 0;
    if (meta & (M_DEAD | M_ABSORBED)) return;
    const SimDev& S = B.sims[sim_of(meta)];
    if (!S.active) return;
    const ModelDev& Mo = B.models[S.model];
    a.S = &S;
    a.Mo = &Mo;
    const uint32_t t = S.step;
    if (t >= S.max_step || S.err) {  // frozen (or failed): kept in place, not advanced
        a.flags = 1u;
        return;
    }
    bool alive = true, emit = false;
    if (meta & M_BOUND) {
        // A release holds its whole warp until the partner is placed, and at
        // 1M agents that warp ends the pass: every load and reservation the
        // release needs is requested as early as its inputs allow.  The
        // partner id is read for every carrier (few agents are in complexes)
        // while the release draw runs.
        const uint32_t par = B.apar[cur][i];
        const ReactionDev& R = Mo.rx[(meta & M_RXN) >> M_RXN_SHIFT];
        const uint4 e = philox(make_uint4(a.id, t, 1u, 0u), S.key0, S.key1);
        if ((uint64_t)e.x < R.thr_rel) {
            const bool ra = meta & M_ROLE_A;
            const int cprod = ra ? R.prod_a : R.prod_b;
            const int hprod = ra ? R.prod_b : R.prod_a;
            meta &= ~(M_BOUND | M_ROLE_A | M_RXN);
            if (hprod >= 0) {  // the partner reappears here and moves on its own
                const uint32_t k = reserve(&ctl->n_extra[parity]);  // in flight during the partner's move
                int4 q = a.p;
                q.w = (int)with_species(meta, (uint32_t)hprod, Mo);
                brownian_move(S, Mo.sp[hprod], B.ztab, q, par, t);
                if (k < B.cap_extras) {
                    const uint32_t key = cell_of(S, q.x, q.y, q.z);
                    const uint32_t rank = atomicAdd(&B.cnt[key], 1u);
                    atomicAdd(&B.tcnt[key / kScanTile * kTileStride], 1u);
                    B.xpm[k] = repack(q, par);
                    B.xrk[k] = rank;  // the scatter finds the cell again from q
                    if (kLive)
                        atomicAdd((unsigned long long*)&live_buffer(B, ctl->epoch)[S.counts_off +
                                                                                   count_slot((uint32_t)q.w, Mo)],
                                  1ull);
                } else {
                    raise_error(ctl, ERR_CAPACITY_EXTRAS, k);
                }
            }
            if (cprod >= 0) meta = with_species(meta, (uint32_t)cprod, Mo);
            else alive = false;
        }
    } else {
        const SpeciesDev& sd = Mo.sp[meta & M_SP];
        if (sd.has_event) {
            const uint4 e = philox(make_uint4(a.id, t, 1u, 0u), S.key0, S.key1);
            if ((uint64_t)e.y < sd.thr_uni) {
                if (sd.uni_to >= 0) meta = with_species(meta, (uint32_t)sd.uni_to, Mo);
                else alive = false;
            } else if ((uint64_t)e.z < sd.thr_emit) {
                emit = true;
            }
        }
    }
    a.p.w = (int)meta;
    if (!alive) return;
    a.flags = 1u | (emit ? 2u : 0u);
    if (Mo.sp[meta & M_SP].M) {
        const uint4 m = philox(make_uint4(a.id, t, 0u, 0u), S.key0, S.key1);
        a.z[0] = __ldg(&B.ztab[m.x >> 16]);
        a.z[1] = __ldg(&B.ztab[m.y >> 16]);
        a.z[2] = __ldg(&B.ztab[m.z >> 16]);
        a.mw = m.w;
        a.flags |= 4u;
    }
}

// Phase 2: apply the step (walls, membranes) and compute the cell key.
__device__ __forceinline__ void move_phase2(MoveState& a) {
    if (!(a.flags & 1u)) return;
    const SimDev& S = *a.S;
    if (a.flags & 4u) {
        const SpeciesDev& sd = a.Mo->sp[(uint32_t)a.p.w & M_SP];
        int32_t x = a.p.x + gauss_step(a.z[0], sd.M);
        int32_t y = a.p.y + gauss_step(a.z[1], sd.M);
        int32_t z = a.p.z + gauss_step(a.z[2], sd.M);
        if (!S.root_sphere) {
            x = fold(x, S.ext);
            y = fold(y, S.ext);
            z = fold(z, S.ext);
        }
        const int c = locate(S, x, y, z);
        bool accept = c >= 0;  // outside the spherical cell: rejected
        if (accept) {
            const uint32_t comp = ((uint32_t)a.p.w & M_COMP) >> M_COMP_SHIFT;
            if ((uint32_t)c != comp) {
                if ((uint64_t)a.mw >= sd.thr_cross) accept = false;  // membrane: rejected
                else a.p.w = (int)(((uint32_t)a.p.w & ~M_COMP) | ((uint32_t)c << M_COMP_SHIFT));
            }
        }
        if (accept) {
            a.p.x = x;
            a.p.y = y;
            a.p.z = z;
        }
    }
    a.key = cell_of(S, a.p.x, a.p.y, a.p.z);
}

// A birth of this step in its simulation's segment of the births buffer:
// (the parent's slot in the moved buffer, its id).  The lanes of one
// simulation reserve together; beyond the simulation's limit its own error
// word is set (the simulation stops, the others go on).
__device__ __noinline__ void reserve_birth(Buffers& B, Ctl* ctl, uint32_t parity, uint32_t sim, uint32_t slot,
                                              uint32_t id) {
    cg::coalesced_group grp = cg::labeled_partition(cg::coalesced_threads(), (int)sim);
    SimDev& S = B.sims[sim];
    uint32_t base = 0;
    if (grp.thread_rank() == 0) base = atomicAdd(&S.nbc[parity], grp.size());
    const uint32_t k = grp.shfl(base, 0) + grp.thread_rank();
    if (k < B.bquota) {
        B.bseg[(size_t)sim * B.bquota + k] = make_uint2(slot, id);
    } else if (atomicCAS(&S.err, 0u, SIM_ERR_BIRTHS) == 0u) {
        S.err_info = k;
        atomicAdd(&ctl->sim_errs, 1u);
    }
}

// Phase 4: results (the histogram rank comes from the atomic between) and births.
__device__ __forceinline__ void move_phase4(Buffers& B, Ctl* ctl, uint32_t cur, uint32_t parity, uint32_t i,
                                            const MoveState& a, uint32_t rank) {
    if (!(a.flags & 1u)) {
        B.rk[i] = kNone;
        return;
    }
    B.rk[i] = rank;  // the scatter finds the cell again from the moved record
    B.pm[cur][i] = repack(a.p, a.id);
    if (a.flags & 2u) reserve_birth(B, ctl, parity, sim_of((uint32_t)a.p.w), i, a.id);
}


template <bool kLive>
__device__ __forceinline__ void move_pass(Buffers& B, uint32_t bid, uint32_t nb) {
    Ctl* ctl = B.ctl;
    const uint32_t cur = ctl->cur;
    const uint32_t n = ctl->n_buf[cur];
    const uint32_t epoch = ctl->epoch, parity = epoch & 1u;
    if (bid == 0 && threadIdx.x == 0) {
        ctl->n_sorted = 0;             // the scan writes the count (if any cell is in use)
        ctl->move_parity = epoch & 1u;  // stable during k_scan, whose bookkeeping advances epoch
    }
    const int4* __restrict__ pm = B.pm[cur];
    // proposal slots touched last step become empty again (the list is short)
    const uint32_t np = ctl->n_props[parity ^ 1u];
    const uint32_t stride = nb * blockDim.x;
    for (uint32_t k = bid * blockDim.x + threadIdx.x; k < np; k += stride) B.acc[B.props[k].y] = kEmpty;
    // threshold monitors add up the records as they stand after t steps (a
    // loop of its own: it keeps the main loop's register count)
    if (ctl->n_monitors)
        for (uint32_t i = bid * blockDim.x + threadIdx.x; i < n; i += stride)
            monitor_record(B, (uint32_t)pm[i].z, kNone);
    // Each warp takes a contiguous range of agents, 32 consecutive ones per
    // iteration (coalesced).  The next 32 records are loaded while these run
    // their chain of dependent table lookups and the histogram atomic.  The
    // range is in cell order from the last step, so its agents stay in one
    // cell tile for long stretches: the warp keeps the tile's count in
    // registers and adds it to the tile counter when the tile changes.
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = nb * (blockDim.x >> 5);
    const uint32_t w = bid * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint32_t len = ((n + warps - 1) / warps + 31u) & ~31u;
    const uint32_t wbeg = min(n, w * len), wend = min(n, wbeg + len);
    // live counts of the step's result (the variant launched while they are
    // on): the moved agents here.  A block's range is contiguous in cell
    // order, so nearly all belong to the simulation of its first agent: a
    // shared histogram for that one.
    constexpr bool count_live = kLive;
    __shared__ uint32_t s_live[kLive ? 512 : 1];
    __shared__ uint32_t s_live_sim;
    if (count_live) {
        for (uint32_t k = threadIdx.x; k < 512; k += blockDim.x) s_live[k] = 0;
        if (threadIdx.x == 0) {
            const uint32_t first = min(n, bid * (blockDim.x >> 5) * len);
            s_live_sim = first < n ? sim_of((uint32_t)pm[first].z) : kNone;
        }
        __syncthreads();
    }
    int4 nx_p = make_int4(0, 0, 0, 0);  // the next packed record
    if (wbeg + lane < wend) nx_p = pm[wbeg + lane];
    uint32_t run_tile = kNone, run_n = 0;  // the same in every lane
    for (uint32_t base = wbeg; base < wend; base += 32) {  // uniform over the warp
        const uint32_t i = base + lane;
        MoveState a;
        a.flags = 0;
        a.p = unpack_rec(nx_p);
        a.id = (uint32_t)nx_p.w;
        if (i + 32 < wend) nx_p = pm[i + 32];
        if (i < wend) {
            move_phase1<kLive>(B, ctl, cur, parity, i, a);
            move_phase2(a);
        }
        const uint32_t rank = (a.flags & 1u) ? atomicAdd(&B.cnt[a.key], 1u) : 0u;
        const uint32_t tile = (a.flags & 1u) ? a.key / kScanTile : kNone;
        const uint32_t live = __ballot_sync(0xFFFFFFFFu, tile != kNone);
        if (live) {
            const uint32_t t0 = __shfl_sync(0xFFFFFFFFu, tile, __ffs(live) - 1);
            const uint32_t same = __ballot_sync(0xFFFFFFFFu, tile == t0);
            if (t0 != run_tile) {
                if (run_n && lane == 0) atomicAdd(&B.tcnt[run_tile * kTileStride], run_n);
                run_tile = t0;
                run_n = 0;
            }
            run_n += __popc(same);
            if (tile != kNone && tile != t0) atomicAdd(&B.tcnt[tile * kTileStride], 1u);
        }
        if (i < wend) move_phase4(B, ctl, cur, parity, i, a, rank);
        if (count_live && (a.flags & 1u)) {
            const uint32_t meta = (uint32_t)a.p.w, slot = count_slot(meta, *a.Mo);
            if (sim_of(meta) == s_live_sim) atomicAdd(&s_live[slot], 1u);
            else atomicAdd((unsigned long long*)&live_buffer(B, epoch)[a.S->counts_off + slot], 1ull);
        }
    }
    if (run_n && lane == 0) atomicAdd(&B.tcnt[run_tile * kTileStride], run_n);
    if (count_live) {
        __syncthreads();
        if (s_live_sim != kNone) {
            uint64_t* L = live_buffer(B, epoch) + B.sims[s_live_sim].counts_off;
            for (uint32_t k = threadIdx.x; k < 512; k += blockDim.x)
                if (s_live[k]) atomicAdd((unsigned long long*)&L[k], (unsigned long long)s_live[k]);
        }
    }
}

// Block size TB (128, 256 or 512 threads; the autotuner's choice) with the
// register budget of 64 per thread, or with kDense 48 (1280 threads per SM:
// five 256-thread blocks instead of four).  More warps in flight pay on
// large batches (16M agents: 502 -> 486 us per step); at 1M agents the
// 64-register pass measured faster (22.5-23.0 against 24.6 us).
template <bool kLive, int TB, bool kDense>
__global__ void __launch_bounds__(TB, (kDense ? 1280 : 1024) / TB) k_move(Buffers B) {
    pdl_wait();
    if (ld_volatile(&B.ctl->err)) return;
    move_pass<kLive>(B, blockIdx.x, gridDim.x);
    pdl_trigger();
}

// ------------------------------------------------------------------------
// Exclusive block scan of one value per thread; returns the thread's
// exclusive prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t wpre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; w++) {
        const uint32_t sw = s_warp[w];
        if (w < warp) wpre += sw;
        tot += sw;
    }
    __syncthreads();  // s_warp may be reused by the caller
    *total = tot;
    return wpre + incl - v;
}

// ------------------------------------------------------------------------
// The cell scan.  The move pass has counted the agents of every cell and of
// every tile of 8192 cells.  Up to kDirectTiles tiles, each k_scan block
// adds up the tile counts before its own range of tiles itself; beyond that
// one block of k_tile_prefix first turns the tile counts into prefixes.
__global__ void __launch_bounds__(1024) k_tile_prefix(Buffers B) {
    __shared__ uint32_t s_warp[32];
    Ctl* ctl = B.ctl;
    pdl_wait();
    if (ld_volatile(&ctl->err)) return;
    const uint32_t n = ctl->n_cells;
    const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t run = 0;
    for (uint32_t base = 0; base < ntiles; base += blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        const uint32_t v = t < ntiles ? B.tcnt[t * kTileStride] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        uint32_t wpre = 0, tot = 0;
        for (int k = 0; k < (int)(blockDim.x / 32); k++) {
            const uint32_t sw = s_warp[k];
            if (k < warp) wpre += sw;
            tot += sw;
        }
        __syncthreads();
        if (t < ntiles) B.tsum[t] = run + wpre + incl - v;
        run += tot;
    }
    if (threadIdx.x == 0) B.tsum[ntiles] = run;
    pdl_trigger();
}

// One scan tile: start[c] = agents in the tiles before + the tile's own
// exclusive prefix; its counts are reset to zero for the next step.  Warp w
// takes the tile's w-th 1024 cells as 8 rows of 128, lane l cells 4l..4l+3
// of each row, so that every load and store of a warp is 512 contiguous
// bytes.  The agents before the tile are `prefix` plus, when pre_n > 0, the
// counts of tiles [pre_first, pre_first + pre_n) added up here after this
// tile's own counts have been requested, so that both sets of loads are in
// flight at once.  Returns the agents before the next tile.
__device__ __forceinline__ uint32_t scan_tile(Buffers& B, uint32_t tile, uint32_t prefix, uint32_t pre_first,
                                              uint32_t pre_n, uint32_t* s_warp) {
    constexpr uint32_t kRows = kScanTile / kThreads / 4;  // rows of 128 cells per warp
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t base = tile * kScanTile + warp * (kScanTile / (kThreads / 32)) + lane * 4;
    uint4* src = reinterpret_cast<uint4*>(B.cnt + base);  // row k at src + 32 k
    uint4 v[kRows];
#pragma unroll
    for (uint32_t k = 0; k < kRows; k++) v[k] = src[32 * k];
    uint32_t pre_v = 0;
    for (uint32_t t = pre_first + threadIdx.x; t < pre_first + pre_n; t += blockDim.x)
        pre_v += B.tcnt[t * kTileStride];
#pragma unroll
    for (uint32_t k = 0; k < kRows; k++) src[32 * k] = make_uint4(0, 0, 0, 0);
    // exclusive prefix of each lane's four cells within the warp's rows
    uint32_t off[kRows], wtot = 0;
#pragma unroll
    for (uint32_t k = 0; k < kRows; k++) {
        const uint32_t r = v[k].x + v[k].y + v[k].z + v[k].w;
        uint32_t incl = r;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        off[k] = wtot + incl - r;
        wtot += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (pre_n) {
        uint32_t pre_total;
        block_exclusive_scan(pre_v, s_warp, &pre_total);
        prefix += pre_total;
    }
    uint32_t total;
    const uint32_t wpre = __shfl_sync(0xFFFFFFFFu, block_exclusive_scan(lane == 0 ? wtot : 0u, s_warp, &total), 0);
    const uint32_t run = prefix + wpre;
    uint4* dst = reinterpret_cast<uint4*>(B.start + base);
#pragma unroll
    for (uint32_t k = 0; k < kRows; k++) {
        uint4 o;
        o.x = run + off[k];
        o.y = o.x + v[k].x;
        o.z = o.y + v[k].y;
        o.w = o.z + v[k].z;
        dst[32 * k] = o;
    }
    return prefix + total;
}

// The step's bookkeeping, run by one extra block of k_scan while the other
// blocks scan (nothing here touches the cell arrays).  The move pass of this
// step (epoch E, parity p) is complete: births reserved per simulation,
// monitor sums added, released partners counted.  For every simulation:
// births placed this step = min(reserved, limit), their prefix over the
// simulations (births are appended after the sorted agents in simulation
// order) and the tiles of segments longer than kBirthTile (the sorter
// blocks derive the same layout), the id of the first child and the new
// next id; the threshold
// monitor's evaluation of the state the step started from; the step counter
// (the step index tau in flight for the proposal search, then advanced
// unless frozen or failed); the live counts' next-id entry.  Then the
// buffer flips (the scatter writes the other buffer), epoch becomes E + 1,
// and the other parity's counters are cleared for the next step.
__device__ void bookkeeping_block(Buffers& B) {
    __shared__ uint32_t s_warp[kThreads / 32];
    Ctl* ctl = B.ctl;
    const uint32_t epoch = ctl->epoch, parity = epoch & 1u;
    const uint32_t n_sims = ctl->n_sims;
    const bool monitors = ctl->n_monitors != 0, live = ctl->live_counts != 0;
    constexpr uint32_t kPer = (kMaxSims + kThreads - 1) / kThreads;  // simulations per thread
    const uint32_t s0 = threadIdx.x * kPer;
    uint32_t nb[kPer], mine = 0;
#pragma unroll
    for (uint32_t k = 0; k < kPer; k++) {
        const uint32_t s = s0 + k;
        nb[k] = 0;
        if (s < n_sims && B.sims[s].active) nb[k] = min(B.sims[s].nbc[parity], B.bquota);
        mine += nb[k];
    }
    uint32_t total;
    uint32_t pre = block_exclusive_scan(mine, s_warp, &total);
    // a segment longer than one tile is ranked through its sorted tiles
    auto tiles_of = [](uint32_t n) { return n > kBirthTile ? (n + kBirthTile - 1) / kBirthTile : 0u; };
    uint32_t tmine = 0;
#pragma unroll
    for (uint32_t k = 0; k < kPer; k++) tmine += tiles_of(nb[k]);
    uint32_t ttotal;
    uint32_t tpre = block_exclusive_scan(tmine, s_warp, &ttotal);
#pragma unroll
    for (uint32_t k = 0; k < kPer; k++) {
        const uint32_t s = s0 + k;
        if (s >= n_sims) break;
        SimDev& S = B.sims[s];
        B.bofs[s] = pre;
        pre += nb[k];
        B.btofs[s] = tpre;
        tpre += tiles_of(nb[k]);
        S.nbt = tiles_of(nb[k]);
        S.nbc[parity ^ 1u] = 0;
        if (!S.active) {
            S.adv = 0;
            continue;
        }
        const uint64_t nid = (uint64_t)S.next_id + nb[k];
        if (nid >= kNone) raise_error(ctl, ERR_ID_SPACE, s);
        S.nb = nb[k];
        S.nid0 = S.next_id;
        S.next_id = (uint32_t)nid;
        if (monitors) monitor_eval(B, s);  // the move pass added up the state this step started from
        const uint32_t adv = S.step < S.max_step && S.err == 0u;
        S.tau = S.step;
        S.adv = adv;
        if (adv) S.step += 1;
        if (live)  // the last entry of a counts vector is the next id
            live_buffer(B, epoch)[S.counts_off + S.n_counts - 1] = S.next_id;
    }
    if (threadIdx.x == 0) {
        B.bofs[n_sims] = total;
        B.btofs[n_sims] = ttotal;
        ctl->nb_total = total;
        ctl->cur ^= 1u;
        ctl->epoch = epoch + 1u;
        ctl->n_extra[parity ^ 1u] = 0;
        ctl->n_props[parity] = 0;
    }
}

// Sorter block j of kSortBlocks in k_scan: every births segment longer than
// kBirthTile is cut into tiles of kBirthTile births (the layout the
// bookkeeping block also derives, for the ranking in k_propose); this block
// sorts tiles j, j + kSortBlocks, ... : the parent ids of the tile ascending
// in shared memory (bitonic network; a short last tile padded with the
// largest id, which no parent has), written to bsrt at the same positions.
// Without a long segment it finds no tile and returns.
__device__ void sorter_block(Buffers& B, uint32_t j, uint32_t* s_keys, uint32_t* s_warp, uint32_t* s_own) {
    Ctl* ctl = B.ctl;
    const uint32_t parity = ctl->move_parity, n_sims = ctl->n_sims;
    constexpr uint32_t kPer = (kMaxSims + kThreads - 1) / kThreads;
    const uint32_t s0 = threadIdx.x * kPer;
    uint32_t tiles[kPer], mine = 0;
#pragma unroll
    for (uint32_t k = 0; k < kPer; k++) {
        const uint32_t s = s0 + k;
        uint32_t nb = 0;
        if (s < n_sims && B.sims[s].active) nb = min(B.sims[s].nbc[parity], B.bquota);
        tiles[k] = nb > kBirthTile ? (nb + kBirthTile - 1) / kBirthTile : 0u;
        mine += tiles[k];
    }
    uint32_t total;
    const uint32_t pre = block_exclusive_scan(mine, s_warp, &total);
    for (uint32_t t = j; t < total; t += kSortBlocks) {
        uint32_t run = pre;
#pragma unroll
        for (uint32_t k = 0; k < kPer; k++) {  // the thread that owns tile t's simulation names it
            if (t >= run && t < run + tiles[k]) {
                s_own[0] = s0 + k;
                s_own[1] = t - run;
            }
            run += tiles[k];
        }
        __syncthreads();
        const uint32_t s = s_own[0], base = s_own[1] * kBirthTile;
        const uint32_t len = min(kBirthTile, min(B.sims[s].nbc[parity], B.bquota) - base);
        const uint2* seg = B.bseg + (size_t)s * B.bquota + base;
        for (uint32_t k = threadIdx.x; k < kBirthTile; k += blockDim.x) s_keys[k] = k < len ? seg[k].y : kNone;
        __syncthreads();
        for (uint32_t size = 2; size <= kBirthTile; size <<= 1)
            for (uint32_t stride = size / 2; stride > 0; stride >>= 1) {
                for (uint32_t i = threadIdx.x; i < kBirthTile / 2; i += blockDim.x) {
                    const uint32_t lo = 2 * stride * (i / stride) + i % stride, hi = lo + stride;
                    const uint32_t a = s_keys[lo], b = s_keys[hi];
                    if ((a > b) == ((lo & size) == 0)) {
                        s_keys[lo] = b;
                        s_keys[hi] = a;
                    }
                }
                __syncthreads();
            }
        uint32_t* out = B.bsrt + (size_t)s * B.bquota + base;
        for (uint32_t k = threadIdx.x; k < len; k += blockDim.x) out[k] = s_keys[k];
        __syncthreads();  // s_keys and s_own are reused by the next tile
    }
}

// k_scan: block b scans a contiguous range of tiles; the agents before the
// range come from the tile counts (or from k_tile_prefix on large grids).
// The block with the last tile writes the total and the sorted-agent count.
// The block after the scan blocks does the step's bookkeeping, the
// kSortBlocks after it sort the tiles of long births segments.
__global__ void __launch_bounds__(kThreads) k_scan(Buffers B) {
    __shared__ uint32_t s_warp[kThreads / 32];
    Ctl* ctl = B.ctl;
    pdl_wait();
    if (ld_volatile(&ctl->err)) return;
    const uint32_t nblk = gridDim.x - 1 - kSortBlocks;
    if (blockIdx.x >= nblk) {
        if (blockIdx.x == nblk) {
            bookkeeping_block(B);
        } else {
            __shared__ uint32_t s_keys[kBirthTile];
            __shared__ uint32_t s_own[2];
            sorter_block(B, blockIdx.x - nblk - 1, s_keys, s_warp, s_own);
        }
        pdl_trigger();
        return;
    }
    const uint32_t n = ctl->n_cells;
    const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
    const uint32_t per = (ntiles + nblk - 1) / nblk;
    const uint32_t t0 = min(ntiles, blockIdx.x * per), t1 = min(ntiles, t0 + per);
    if (t0 < t1) {
        const bool direct = ntiles <= kDirectTiles;
        uint32_t before = direct ? 0u : B.tsum[t0];
        for (uint32_t t = t0; t < t1; t++)
            before = scan_tile(B, t, before, 0, (direct && t == t0) ? t0 : 0, s_warp);
        if (t1 == ntiles && threadIdx.x == 0) {
            B.start[n] = before;  // cells past n are empty
            ctl->n_sorted = before;
        }
    }
    pdl_trigger();
}

// ------------------------------------------------------------------------
// k_scatter: every live agent (and every released partner) to its slot
// start[cell] + rank in the other buffer.  Each thread moves four agents,
// issuing all loads before the dependent start[] gathers.
constexpr int kScatterILP = 4;

__device__ __forceinline__ void scatter_pass(Buffers& B, uint32_t bid, uint32_t nb) {
    Ctl* ctl = B.ctl;
    // the bookkeeping has flipped the buffers: the moved agents are in cur ^ 1
    const uint32_t nxt = ctl->cur, cur = nxt ^ 1u;
    const uint32_t epoch = ctl->epoch, parity = (epoch - 1u) & 1u;
    const uint32_t n_in = ctl->n_buf[cur], total = n_in + ctl->n_extra[parity];
    // the scan has read this step's tile counts: zero them for the next step
    const uint32_t ntiles = (ctl->n_cells + kScanTile - 1) / kScanTile;
    for (uint32_t t = bid * blockDim.x + threadIdx.x; t < ntiles; t += nb * blockDim.x) B.tcnt[t * kTileStride] = 0;
    if (ctl->live_counts) {  // the live counts the next step fills (the last step's were read by now)
        uint64_t* L = live_buffer(B, epoch);
        const uint32_t n_live = ctl->n_sims * 512u;
        for (uint32_t k = bid * blockDim.x + threadIdx.x; k < n_live; k += nb * blockDim.x) L[k] = 0;
    }
    const uint32_t stride = nb * blockDim.x;
    for (uint32_t j0 = bid * blockDim.x + threadIdx.x; j0 < total; j0 += kScatterILP * stride) {
        uint32_t rk[kScatterILP];
        int4 p[kScatterILP];  // packed records
        uint32_t par[kScatterILP];
#pragma unroll
        for (int u = 0; u < kScatterILP; u++) {
            const uint32_t j = j0 + u * stride;
            rk[u] = kNone;
            par[u] = kNone;
            if (j < n_in) {
                rk[u] = B.rk[j];
                p[u] = B.pm[cur][j];
            } else if (j < total) {
                const uint32_t k = j - n_in;
                rk[u] = B.xrk[k];
                p[u] = B.xpm[k];
            }
        }
        // the cell comes from the moved record, as the move pass computed it
        uint32_t dest[kScatterILP];
#pragma unroll
        for (int u = 0; u < kScatterILP; u++) {
            dest[u] = kNone;
            if (rk[u] == kNone) continue;
            const SimDev& S = B.sims[sim_of((uint32_t)p[u].z)];
            const int4 q = unpack_rec(p[u]);
            dest[u] = B.start[cell_of(S, q.x, q.y, q.z)] + rk[u];
            // the partner id only for carriers (few), requested beside the start[] gather
            if (((uint32_t)p[u].z & M_BOUND) && j0 + u * stride < n_in) par[u] = B.apar[cur][j0 + u * stride];
        }
#pragma unroll
        for (int u = 0; u < kScatterILP; u++) {
            if (dest[u] == kNone) continue;
            if (dest[u] >= B.cap_agents) {
                raise_error(ctl, ERR_CAPACITY_AGENTS, dest[u]);
                continue;
            }
            const uint32_t meta = (uint32_t)p[u].z;
            B.pm[nxt][dest[u]] = p[u];
            B.pflag[dest[u]] = (meta & (M_PROP | M_BOUND)) == M_PROP;
            if (meta & M_BOUND) B.apar[nxt][dest[u]] = par[u];
        }
    }
}

// Last simulation s of [0, n) with ofs[s] <= v (ofs ascending, ofs[0] = 0 <= v).
__device__ __forceinline__ uint32_t last_at_most(const uint32_t* ofs, uint32_t n, uint32_t v) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (ofs[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int TB>
__global__ void __launch_bounds__(TB) k_scatter(Buffers B) {
    pdl_wait();
    if (ld_volatile(&B.ctl->err)) return;
    scatter_pass(B, blockIdx.x, gridDim.x);
    pdl_trigger();
}

// ------------------------------------------------------------------------
// One candidate q (sorted index gj) for proposer p: keep the nearest eligible
// partner by (dist^2, id); the pair draw is taken only when it could win.
struct Best {
    uint64_t key = kEmpty;
    uint32_t target = kNone;
};

__device__ __forceinline__ void consider(const SimDev& S, const ModelDev& Mo, const int4& p, uint32_t meta,
                                         uint32_t sp, uint64_t mask, int rmax, uint32_t ida, const int4& qr,
                                         uint32_t gj, uint32_t t, Best& best) {
    // cheap rejections first: almost every candidate is beyond every radius
    const int4 q = unpack_rec(qr);
    const int dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
    if (abs(dx) > rmax || abs(dy) > rmax || abs(dz) > rmax) return;
    const uint32_t mq = (uint32_t)qr.z;
    if (mq & M_BOUND) return;
    if ((mq ^ meta) & M_COMP) return;
    const uint32_t spb = mq & M_SP;
    if (!((mask >> spb) & 1ull)) return;
    const ReactionDev& R = Mo.rx[Mo.rx_of[sp][spb]];
    if (abs(dx) > R.R || abs(dy) > R.R || abs(dz) > R.R) return;
    const uint32_t d2 = (uint32_t)(dx * dx) + (uint32_t)(dy * dy) + (uint32_t)(dz * dz);
    if (d2 > R.R2) return;
    const uint32_t idb = (uint32_t)qr.w;
    const uint64_t key = (uint64_t)d2 << 32 | idb;
    if (key >= best.key) return;  // cannot win: the draw is not needed
    const uint32_t lo = min(ida, idb), hi = max(ida, idb);
    const uint4 u = philox(make_uint4(lo, hi, t, 1u), S.key0, S.key1);
    if ((uint64_t)u.x >= R.thr_bind) return;
    best.key = key;
    best.target = gj;
}

__device__ __forceinline__ void claim(Buffers& B, const Best& best, uint32_t ida, uint32_t gi, uint32_t parity) {
    if (best.target == kNone) return;
    atomicMin((unsigned long long*)&B.acc[best.target], (unsigned long long)((best.key & 0xFFFFFFFF00000000ull) | ida));
    const uint32_t k = reserve(&B.ctl->n_props[parity]);  // k < capacity: at most one proposal per agent
    B.props[k] = make_uint2(gi, best.target);
}

// ------------------------------------------------------------------------
// k_propose: every free agent of a proposing species (compacted per block
// from 1024 consecutive sorted agents) scans the cells that intersect the box [p - rmax, p + rmax] (rmax: its largest contact radius)
// -- one or two cells per axis, x-consecutive cells forming one contiguous
// range of the cell-sorted array -- keeps the nearest eligible partner by
// (dist^2, id) and claims it with atomicMin.  Any partner within a contact
// radius lies inside that box, so the result equals the 27-cell search.
// One chunk of sorted agents [base, base + chunk): its free agents of
// proposing species are compacted into s_list, then each searches its box.
__device__ __forceinline__ void propose_chunk(Buffers& B, uint32_t base, uint32_t n, uint32_t parity,
                                              uint32_t* s_list, uint32_t* s_n) {
    const uint32_t cur = B.ctl->cur;  // the sorted buffer (flipped by this step's bookkeeping)
    const int4* __restrict__ pm = B.pm[cur];
    const uint32_t* __restrict__ start = B.start;
    const uint32_t chunk = B.propose_chunk;
    // each thread takes chunk / 256 consecutive flags (4, 8 or 16 bytes, read
    // as whole words, all requested at once) and places its proposers after
    // those of the threads before it (order within the list is free)
    const uint32_t per = chunk / kThreads, i0 = base + threadIdx.x * per;
    const uint32_t* fw = reinterpret_cast<const uint32_t*>(B.pflag + i0);  // i0 % 4 == 0
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 4; k++)
        if ((uint32_t)k < per / 4 && i0 + 4 * k < n) w[k] = fw[k];
#pragma unroll
    for (int k = 0; k < 4; k++) {  // flags past n are not agents of this step
        const uint32_t first = i0 + 4 * k;
        if (first < n && n - first < 4) w[k] &= (1u << (8 * (n - first))) - 1u;
    }
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) mine += __popc(w[k]);  // flags are 0 or 1 bytes
    uint32_t total;
    uint32_t pos = block_exclusive_scan(mine, reinterpret_cast<uint32_t*>(s_n) + 1, &total);
#pragma unroll
    for (int k = 0; k < 4; k++)
        for (uint32_t x = w[k]; x; x &= x - 1) s_list[pos++] = i0 + 4 * k + (__ffs(x) - 1) / 8;
    __syncthreads();
    const uint32_t np = total;
    // the next proposer's record is requested while this one searches
    uint32_t gi_n = threadIdx.x < np ? s_list[threadIdx.x] : 0u;
    int4 p_n = threadIdx.x < np ? pm[gi_n] : make_int4(0, 0, 0, 0);
    for (uint32_t k = threadIdx.x; k < np; k += blockDim.x) {
        const uint32_t gi = gi_n;
        const int4 p = unpack_rec(p_n);
        const uint32_t ida = (uint32_t)p_n.w;
        if (k + blockDim.x < np) {
            gi_n = s_list[k + blockDim.x];
            p_n = pm[gi_n];
        }
        const uint32_t meta = (uint32_t)p.w;
        const SimDev& S = B.sims[sim_of(meta)];
        if (!S.adv) continue;  // frozen or failed simulation
        const ModelDev& Mo = B.models[S.model];
        const uint32_t sp = meta & M_SP;
        const uint64_t mask = Mo.sp[sp].partner_mask;
        const int rmax = Mo.sp[sp].rmax;
        const int g = (int)S.g, sh = (int)S.shift;
        const int xlo = max((p.x - rmax) >> sh, 0), xhi = min((p.x + rmax) >> sh, g - 1);
        const int ylo = max((p.y - rmax) >> sh, 0), yhi = min((p.y + rmax) >> sh, g - 1);
        const int zlo = max((p.z - rmax) >> sh, 0), zhi = min((p.z + rmax) >> sh, g - 1);
        Best best;
        // x-consecutive cells of one (z, y) row form one contiguous range of
        // the sorted array, walked one candidate record at a time
        auto walk = [&](uint32_t a, uint32_t b) {
            for (uint32_t j = a; j < b; j++)
                if (j != gi) consider(S, Mo, p, meta, sp, mask, rmax, ida, pm[j], j, S.tau, best);
        };
        if (zhi - zlo <= 1 && yhi - ylo <= 1) {
            // the usual box (2 * rmax below the cell edge): at most 2 x 2 rows,
            // whose bounds are all requested at once
            uint32_t ra[4], rb[4];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int zz = zlo + (r >> 1), yy = ylo + (r & 1);
                const bool in = zz <= zhi && yy <= yhi;
                const uint32_t row = S.cell_off + ((uint32_t)min(zz, zhi) * g + (uint32_t)min(yy, yhi)) * g;
                ra[r] = in ? start[row + xlo] : 0u;
                rb[r] = in ? start[row + xhi + 1] : 0u;
            }
            // the four ranges walked as one sequence of candidates (the same
            // order), so that a warp waits for its longest total, not for the
            // longest range of each row in turn
            const uint32_t e0 = rb[0] - ra[0], e1 = e0 + rb[1] - ra[1], e2 = e1 + rb[2] - ra[2];
            // the proposer's own slot (always in one of the ranges: its cell is
            // in its box) is left out of the sequence
            const uint32_t self = gi >= ra[0] && gi < rb[0]   ? gi - ra[0]
                                  : gi >= ra[1] && gi < rb[1] ? e0 + (gi - ra[1])
                                  : gi >= ra[2] && gi < rb[2] ? e1 + (gi - ra[2])
                                  : gi >= ra[3] && gi < rb[3] ? e2 + (gi - ra[3])
                                                              : kNone;
            const uint32_t total = e2 + rb[3] - ra[3] - (self != kNone ? 1u : 0u);
            auto cand = [&](uint32_t t) -> uint32_t {
                t += t >= self;
                return t < e0 ? ra[0] + t : t < e1 ? ra[1] + (t - e0) : t < e2 ? ra[2] + (t - e1) : ra[3] + (t - e2);
            };
            // the next candidate's record is requested while this one is examined
            uint32_t jn = total ? cand(0) : 0u;
            int4 qn = total ? pm[jn] : make_int4(0, 0, 0, 0);
            for (uint32_t t = 0; t < total; t++) {
                const uint32_t j = jn;
                const int4 q = qn;
                if (t + 1 < total) {
                    jn = cand(t + 1);
                    qn = pm[jn];
                }
                consider(S, Mo, p, meta, sp, mask, rmax, ida, q, j, S.tau, best);
            }
        } else {
            // a box wider than half a cell can meet 3 cells per axis (a cell is
            // never smaller than a contact radius): up to 3 x 3 rows
            for (int zz = zlo; zz <= zhi; zz++)
                for (int yy = ylo; yy <= yhi; yy++) {
                    const uint32_t row = S.cell_off + ((uint32_t)zz * g + (uint32_t)yy) * g;
                    walk(start[row + xlo], start[row + xhi + 1]);
                }
        }
        claim(B, best, ida, gi, parity);
    }
    __syncthreads();  // s_list and s_n are reused by the next chunk
}

// Number of entries below x in the sorted keys[0, n) (binary search).
__device__ __forceinline__ uint32_t count_below(const uint32_t* keys, uint32_t n, uint32_t x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        if (keys[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Births of this step (P6): each simulation's children, from its segment of
// the births buffer, get ids nid0 + rank, the rank ordering them by parent
// id (unique: at most one child per parent per step), and are appended
// after the sorted agents, simulation after simulation.  A child is its
// parent's moved record (end of P2: place and compartment) with the
// parent's emitted species; it first acts at the next step.  Thread g of
// the grid places the g-th birth of the step; the simulation it belongs to
// comes from the births prefix (bofs, written by the bookkeeping block),
// searched in shared memory.  The rank: in a segment of at most kBirthTile
// births, by comparing with every other birth of the segment; in a longer
// one, as the sum over its tiles (sorted by the scatter) of the parent ids
// below this one, by binary search -- the tiles staged in shared memory
// when the block's threads share the simulation (the usual case: a long
// segment fills whole blocks), else searched in global memory.
__device__ __noinline__ void place_births(Buffers& B, uint32_t cur, uint32_t nbt, uint32_t ns,
                                             uint32_t* s_bofs, uint32_t* s_tile) {
    Ctl* ctl = B.ctl;
    const uint32_t n_sims = ctl->n_sims;
    for (uint32_t s = threadIdx.x; s <= n_sims; s += blockDim.x) s_bofs[s] = B.bofs[s];
    __syncthreads();
    const uint32_t src = cur ^ 1u;  // the moved (unsorted) buffer holds the parents' records
    uint64_t* live = ctl->live_counts ? live_buffer(B, ctl->epoch - 1u) : nullptr;
    for (uint32_t g0 = blockIdx.x * blockDim.x; g0 < nbt; g0 += gridDim.x * blockDim.x) {  // block-uniform
        const uint32_t g = g0 + threadIdx.x;
        const bool valid = g < nbt;
        const uint32_t s = valid ? last_at_most(s_bofs, n_sims, g) : kNone;
        const uint32_t s_blk = last_at_most(s_bofs, n_sims, g0);  // the block's first birth's
        const uint32_t k = valid ? g - s_bofs[s] : 0u;
        const uint2* seg = valid ? B.bseg + (size_t)s * B.bquota : nullptr;
        const uint32_t pid = valid ? seg[k].y : 0u;
        uint32_t rank = 0;
        // long segment of the block's simulation: its sorted tiles through shared memory
        const uint32_t tiles_blk = B.sims[s_blk].nbt, nb_blk = s_bofs[s_blk + 1] - s_bofs[s_blk];
        for (uint32_t t = 0; t < tiles_blk; t++) {
            const uint32_t base = t * kBirthTile, len = min(kBirthTile, nb_blk - base);
            const uint32_t* tile = B.bsrt + (size_t)s_blk * B.bquota + base;
            for (uint32_t q = threadIdx.x; q < len; q += blockDim.x) s_tile[q] = tile[q];
            __syncthreads();
            if (s == s_blk) rank += count_below(s_tile, len, pid);
            __syncthreads();
        }
        if (!valid) continue;
        const uint32_t nb = s_bofs[s + 1] - s_bofs[s];
        const uint32_t tiles = B.sims[s].nbt;
        if (tiles == 0) {
            rank = 0;
            const uint4* seg4 = reinterpret_cast<const uint4*>(seg);  // bquota is even: 16-byte aligned
            for (uint32_t j = 0; j < nb / 2; j++) {
                const uint4 v = seg4[j];
                rank += (v.y < pid) + (v.w < pid);
            }
            if (nb & 1u) rank += seg[nb - 1].y < pid;
        } else if (s != s_blk) {  // (a long segment starting inside this block)
            rank = 0;
            for (uint32_t t = 0; t < tiles; t++) {
                const uint32_t base = t * kBirthTile;
                rank += count_below(B.bsrt + (size_t)s * B.bquota + base, min(kBirthTile, nb - base), pid);
            }
        }
        const SimDev& S = B.sims[s];
        const ModelDev& Mo = B.models[S.model];
        int4 q = B.pm[src][seg[k].x];  // the parent's packed record: its place
        const uint32_t meta = (uint32_t)q.z;
        q.z = (int)with_species(meta & ~(M_RXN | M_BOUND | M_ROLE_A), (uint32_t)Mo.sp[meta & M_SP].emit, Mo);
        q.w = (int)(S.nid0 + rank);
        const uint32_t dst = ns + s_bofs[s] + rank;
        B.pm[cur][dst] = q;
        if (live) atomicAdd((unsigned long long*)&live[S.counts_off + count_slot((uint32_t)q.z, Mo)], 1ull);
    }
}

__global__ void __launch_bounds__(kThreads) k_propose(Buffers B) {
    extern __shared__ uint32_t s_list[];  // B.propose_chunk entries, max sims + 1 birth offsets, a births tile
    __shared__ uint32_t s_n[1 + kThreads / 32];  // scratch of the compaction's block scan
    pdl_wait();
    Ctl* ctl = B.ctl;
    if (ld_volatile(&ctl->err)) return;
    const uint32_t n = ctl->n_sorted, nbt = ctl->nb_total;
    const uint32_t cur = ctl->cur, parity = (ctl->epoch - 1u) & 1u;
    const bool fits = (uint64_t)n + nbt <= B.cap_agents;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (fits) ctl->n_buf[cur] = n + nbt;
        else raise_error(ctl, ERR_CAPACITY_AGENTS, n + nbt);
    }
    const uint32_t chunk = B.propose_chunk;
    for (uint32_t base = blockIdx.x * chunk; base < n; base += gridDim.x * chunk)
        propose_chunk(B, base, n, parity, s_list, s_n);
    if (nbt && fits) place_births(B, cur, nbt, n, s_list + chunk, s_list + chunk + B.max_sims + 1);
    pdl_trigger();
}

// ------------------------------------------------------------------------
// k_accept: walks the proposal list; edge i -> j is final iff j's slot holds
// i's id and nobody proposed to i.  Final edges are disjoint, so each is
// applied without further synchronisation.
__device__ __forceinline__ void accept_pass(Buffers& B, uint32_t bid, uint32_t nb) {
    Ctl* ctl = B.ctl;
    const uint32_t cur = ctl->cur;  // the sorted buffer
    const uint32_t epoch = ctl->epoch, parity = (epoch - 1u) & 1u;
    const uint32_t np = ctl->n_props[parity];
    uint64_t* live = ctl->live_counts ? live_buffer(B, epoch - 1u) : nullptr;
    int4* __restrict__ pm = B.pm[cur];
    uint32_t* __restrict__ apar = B.apar[cur];
    for (uint32_t k = bid * blockDim.x + threadIdx.x; k < np; k += nb * blockDim.x) {
        const uint2 e = B.props[k];
        const uint32_t i = e.x, j = e.y;
        // the (meta, id) words of both records are loaded with the slots (one round trip less)
        uint2* wa = reinterpret_cast<uint2*>(&pm[i]) + 1;
        uint2* wb = reinterpret_cast<uint2*>(&pm[j]) + 1;
        const uint64_t kb = B.acc[j];
        const uint64_t ka = B.acc[i];
        const uint2 ra = *wa, rb = *wb;
        const uint32_t ida = ra.y;
        uint32_t ma = ra.x, mb = rb.x;
        if ((uint32_t)kb != ida || ka != kEmpty) continue;
        const uint32_t ma0 = ma, mb0 = mb;
        const SimDev& S = B.sims[sim_of(ma)];
        const ModelDev& Mo = B.models[S.model];
        const uint32_t r = Mo.rx_of[ma & M_SP][mb & M_SP];
        const ReactionDev& R = Mo.rx[r];
        if (R.kind == 0) {  // CONVERT
            ma = R.prod_a >= 0 ? with_species(ma, (uint32_t)R.prod_a, Mo) : ma | M_DEAD;
            mb = R.prod_b >= 0 ? with_species(mb, (uint32_t)R.prod_b, Mo) : mb | M_DEAD;
        } else if (R.carrier_a) {  // BIND, a carries b
            ma |= M_BOUND | M_ROLE_A | (r << M_RXN_SHIFT);
            apar[i] = rb.y;
            mb |= M_ABSORBED;
        } else {  // BIND, b carries a
            mb |= M_BOUND | (r << M_RXN_SHIFT);
            apar[j] = ida;
            ma |= M_ABSORBED;
        }
        reinterpret_cast<uint32_t*>(wa)[0] = ma;
        reinterpret_cast<uint32_t*>(wb)[0] = mb;
        if (live) {  // the move pass counted both as they were
            unsigned long long* L = (unsigned long long*)live + S.counts_off;
            atomicAdd(L + count_slot(ma0, Mo), ~0ull);
            atomicAdd(L + count_slot(mb0, Mo), ~0ull);
            if (!(ma & (M_DEAD | M_ABSORBED))) atomicAdd(L + count_slot(ma, Mo), 1ull);
            if (!(mb & (M_DEAD | M_ABSORBED))) atomicAdd(L + count_slot(mb, Mo), 1ull);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_accept(Buffers B) {
    pdl_wait();
    if (ld_volatile(&B.ctl->err)) return;
    accept_pass(B, blockIdx.x, gridDim.x);
    pdl_trigger();
}

// ------------------------------------------------------------------------
// k_init: initial placement of simulation `sim` (ids 0..n0-1, species-major)
// by rejection: uniform integer coordinates from Philox(id, attempt, 0, 2)
// until the point lies in the species' compartment.
__global__ void __launch_bounds__(kThreads) k_init(Buffers B, uint32_t sim, uint32_t base, uint32_t n0,
                                                   const uint32_t* __restrict__ species_end, uint32_t n_sp) {
    Ctl* ctl = B.ctl;
    const uint32_t cur = ctl->cur;
    const SimDev& S = B.sims[sim];
    const ModelDev& Mo = B.models[S.model];
    const uint64_t span = (uint64_t)S.ext + 1;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n0; k += gridDim.x * blockDim.x) {
        uint32_t sp = 0;
        while (sp + 1 < n_sp && species_end[sp] <= k) sp++;
        const int want = (int)Mo.sp[sp].init_comp;
        bool placed = false;
        int32_t x = 0, y = 0, z = 0;
        for (uint32_t attempt = 0; attempt < (1u << 24) && !placed; attempt++) {
            const uint4 w = philox(make_uint4(k, attempt, 0u, 2u), S.key0, S.key1);
            x = (int32_t)(((uint64_t)w.x * span) >> 32);
            y = (int32_t)(((uint64_t)w.y * span) >> 32);
            z = (int32_t)(((uint64_t)w.z * span) >> 32);
            placed = locate(S, x, y, z) == want;
        }
        if (!placed) raise_error(ctl, ERR_PLACEMENT, k);
        const uint32_t meta = with_species((sim << M_SIM_SHIFT) | ((uint32_t)want << M_COMP_SHIFT), sp, Mo);
        B.pm[cur][base + k] = pack_rec(x, y, z, meta, k);
    }
}

// ------------------------------------------------------------------------
// k_observe: per-simulation counts (free by species and compartment, bound
// complexes by reaction) and, optionally, the order-independent digest
// (wrapping sum of a hash of every agent record, hidden partners included).
// Each block owns one contiguous range of the cell-sorted array, so almost
// all of its agents belong to one simulation: those are counted in a
// shared-memory histogram and flushed with one atomic per bin.
__device__ __forceinline__ void observe_one(Buffers& B, uint32_t cur, uint32_t i, const int4& pr, int32_t only_sim,
                                            int want_digest, uint32_t sim0, uint32_t* sh) {
    const uint32_t meta = (uint32_t)pr.z;
    const int4 p = unpack_rec(pr);
    if (meta & (M_DEAD | M_ABSORBED)) return;
    const uint32_t s = sim_of(meta);
    if (only_sim >= 0 && s != (uint32_t)only_sim) return;
    const SimDev& S = B.sims[s];
    if (!S.active) return;
    const ModelDev& Mo = B.models[S.model];
    const uint32_t sp = meta & M_SP, comp = (meta & M_COMP) >> M_COMP_SHIFT;
    uint32_t slot;
    uint64_t h = 0;
    if (meta & M_BOUND) {
        const uint32_t r = (meta & M_RXN) >> M_RXN_SHIFT;
        slot = Mo.n_sp * Mo.n_comp + r;
        if (want_digest) {
            const ReactionDev& R = Mo.rx[r];
            const uint32_t id = (uint32_t)pr.w;
            const uint32_t par = B.apar[cur][i];
            const bool ra = meta & M_ROLE_A;
            h = record_hash(id, sp, comp, 1u | (ra ? 4u : 0u), r, p.x, p.y, p.z, par);
            h += record_hash(par, ra ? R.b : R.a, comp, 2u | (ra ? 0u : 4u), r, p.x, p.y, p.z, id);
        }
    } else {
        slot = sp * Mo.n_comp + comp;
        if (want_digest) h = record_hash((uint32_t)pr.w, sp, comp, 0u, 0xFFu, p.x, p.y, p.z, kNone);
    }
    if (s == sim0) atomicAdd(&sh[slot], 1u);
    else atomicAdd((unsigned long long*)&B.counts[S.counts_off + slot], 1ull);
    if (want_digest) {
        // reduce over the threads of the same simulation: one atomic each
        cg::coalesced_group grp = cg::labeled_partition(cg::coalesced_threads(), (int)s);
        const uint64_t sum = cg::reduce(grp, h, cg::plus<uint64_t>());
        if (grp.thread_rank() == 0) atomicAdd((unsigned long long*)&B.digests[s], (unsigned long long)sum);
    }
}

constexpr int kObserveILP = 4;

__global__ void __launch_bounds__(kThreads) k_observe(Buffers B, int32_t only_sim, int want_digest) {
    __shared__ uint32_t sh[512];
    __shared__ uint32_t s_sim;
    Ctl* ctl = B.ctl;
    const uint32_t cur = ctl->cur;
    const uint32_t n = ctl->n_buf[cur];
    const uint32_t chunk = ((n + gridDim.x - 1) / gridDim.x + kThreads - 1) / kThreads * kThreads;
    const uint32_t begin = blockIdx.x * chunk;
    const uint32_t end = min(n, begin + chunk);
    for (uint32_t k = threadIdx.x; k < 512; k += blockDim.x) sh[k] = 0;
    if (threadIdx.x == 0) {
        uint32_t s0 = kNone;
        if (only_sim >= 0) s0 = (uint32_t)only_sim;
        else if (begin < end) s0 = sim_of((uint32_t)B.pm[cur][begin].z);
        s_sim = s0;
    }
    __syncthreads();
    const uint32_t sim0 = s_sim;
    // several records per thread, all requested before any is examined
    for (uint32_t i0 = begin + threadIdx.x; i0 < end; i0 += kObserveILP * blockDim.x) {
        int4 p[kObserveILP];
#pragma unroll
        for (int u = 0; u < kObserveILP; u++) {
            const uint32_t i = i0 + u * blockDim.x;
            p[u] = i < end ? B.pm[cur][i] : make_int4(0, 0, (int)M_DEAD, 0);
        }
#pragma unroll
        for (int u = 0; u < kObserveILP; u++) observe_one(B, cur, i0 + u * blockDim.x, p[u], only_sim, want_digest, sim0, sh);
    }
    __syncthreads();
    if (sim0 != kNone) {
        const SimDev& S = B.sims[sim0];
        for (uint32_t k = threadIdx.x; k < S.n_counts; k += blockDim.x)
            if (sh[k]) atomicAdd((unsigned long long*)&B.counts[S.counts_off + k], (unsigned long long)sh[k]);
    }
    if (blockIdx.x == 0) {
        const uint32_t n_sims = ctl->n_sims;
        for (uint32_t s = threadIdx.x; s < n_sims; s += blockDim.x) {
            if (only_sim >= 0 && s != (uint32_t)only_sim) continue;
            const SimDev& S = B.sims[s];
            if (!S.active) continue;
            B.counts[S.counts_off + S.n_counts - 1] = S.next_id;
            if (want_digest)
                atomicAdd((unsigned long long*)&B.digests[s],
                          (unsigned long long)fmix64((uint64_t)S.step | (uint64_t)S.next_id << 32));
        }
    }
}

// k_monitor_pass / k_monitor_eval: between steps, the same sum for one
// simulation's current state (a state no step has evaluated yet, e.g. the
// last one), then its evaluation.
__global__ void __launch_bounds__(kThreads) k_monitor_pass(Buffers B, uint32_t sim) {
    Ctl* ctl = B.ctl;
    const uint32_t cur = ctl->cur;
    const uint32_t n = ctl->n_buf[cur];
    const SimDev& S = B.sims[sim];
    if (!S.active || !mon_due(B.mons[sim], S.step)) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        monitor_record(B, (uint32_t)B.pm[cur][i].z, sim);
}

__global__ void k_monitor_eval(Buffers B, uint32_t sim) { monitor_eval(B, sim); }

// k_compact: between steps, copy the agents of active simulations (dropping
// those of retired ones) to the other buffer; storage order is free.  The
// host has zeroed ctl.n_compact, which counts the agents kept.
__global__ void __launch_bounds__(kThreads) k_compact(Buffers B) {
    Ctl* ctl = B.ctl;
    const uint32_t cur = ctl->cur, nxt = cur ^ 1u;
    const uint32_t n = ctl->n_buf[cur];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int4 p = B.pm[cur][i];
        const uint32_t meta = (uint32_t)p.z;
        if (meta & (M_DEAD | M_ABSORBED)) continue;
        if (!B.sims[sim_of(meta)].active) continue;
        const uint32_t k = reserve(&ctl->n_compact);
        B.pm[nxt][k] = p;
        if (meta & M_BOUND) B.apar[nxt][k] = B.apar[cur][i];
    }
}

// k_dump: one record per agent of `sim` (two for a complex), unordered.
__global__ void __launch_bounds__(kThreads) k_dump(Buffers B, int32_t sim, uint4* out_lo, uint2* out_hi,
                                                   uint32_t cap) {
    Ctl* ctl = B.ctl;
    const uint32_t cur = ctl->cur;
    const uint32_t n = ctl->n_buf[cur];
    const SimDev& S = B.sims[sim];
    const ModelDev& Mo = B.models[S.model];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int4 pr = B.pm[cur][i];
        const uint32_t meta = (uint32_t)pr.z;
        if (meta & (M_DEAD | M_ABSORBED)) continue;
        if (sim_of(meta) != (uint32_t)sim) continue;
        const int4 p = unpack_rec(pr);
        const uint32_t sp = meta & M_SP, comp = (meta & M_COMP) >> M_COMP_SHIFT;
        const uint32_t id = (uint32_t)pr.w;
        const bool bound = meta & M_BOUND;
        const uint32_t k = atomicAdd(&ctl->dump_n, bound ? 2u : 1u);
        if (k + (bound ? 2u : 1u) > cap) continue;  // host sees dump_n > cap
        if (bound) {
            const uint32_t r = (meta & M_RXN) >> M_RXN_SHIFT;
            const bool ra = meta & M_ROLE_A;
            const uint32_t par = B.apar[cur][i];
            const uint32_t hs = ra ? Mo.rx[r].b : Mo.rx[r].a;
            out_lo[k] = make_uint4(id, sp | comp << 8 | (1u | (ra ? 4u : 0u)) << 16 | r << 24,
                                   (uint32_t)p.x, (uint32_t)p.y);
            out_hi[k] = make_uint2((uint32_t)p.z, par);
            out_lo[k + 1] = make_uint4(par, hs | comp << 8 | (2u | (ra ? 0u : 4u)) << 16 | r << 24,
                                       (uint32_t)p.x, (uint32_t)p.y);
            out_hi[k + 1] = make_uint2((uint32_t)p.z, id);
        } else {
            out_lo[k] = make_uint4(id, sp | comp << 8 | 0xFFu << 24, (uint32_t)p.x, (uint32_t)p.y);
            out_hi[k] = make_uint2((uint32_t)p.z, kNone);
        }
    }
}

__global__ void k_debug_philox(const uint4* ctr, const uint2* key, uint4* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = philox(ctr[i], key[i].x, key[i].y);
}

}  // namespace

// ------------------------------------------------------------------------
// Launch with programmatic stream serialisation: the kernel may begin
// launching while the previous kernel in the stream drains (it waits in
// pdl_wait before touching any data).
template <typename Kernel>
cudaError_t launch_pdl(Kernel kernel, int grid, cudaStream_t s, const Buffers& B, size_t smem = 0,
                       int threads = kThreads) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, B);
}

// Dynamic shared memory of k_propose: the chunk's proposer list, the births
// prefix of every simulation slot, then one sorted births tile.
size_t propose_smem(const Buffers& B) { return 4 * ((size_t)B.propose_chunk + B.max_sims + 1 + kBirthTile); }

namespace {
using StepKernel = void (*)(Buffers);
// k_move (without, with live counts) and k_scatter for a block size and
// register budget
struct MoveKernels {
    StepKernel move, move_live, scatter;
};
MoveKernels move_kernels(int threads, bool dense) {
    if (threads == 128)
        return dense ? MoveKernels{k_move<false, 128, true>, k_move<true, 128, true>, k_scatter<128>}
                     : MoveKernels{k_move<false, 128, false>, k_move<true, 128, false>, k_scatter<128>};
    if (threads == 512)
        return dense ? MoveKernels{k_move<false, 512, true>, k_move<true, 512, true>, k_scatter<512>}
                     : MoveKernels{k_move<false, 512, false>, k_move<true, 512, false>, k_scatter<512>};
    return dense ? MoveKernels{k_move<false, 256, true>, k_move<true, 256, true>, k_scatter<256>}
                 : MoveKernels{k_move<false, 256, false>, k_move<true, 256, false>, k_scatter<256>};
}
}  // namespace

bool valid_move_threads(int threads) { return threads == 128 || threads == 256 || threads == 512; }

int move_blocks_per_sm(int threads, bool dense, bool live) {
    int n = 0;
    const MoveKernels mk = move_kernels(threads, dense);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, live ? mk.move_live : mk.move, threads, 0) !=
            cudaSuccess ||
        n < 1)
        n = 1024 / threads;
    return n;
}

int scatter_blocks_per_sm(int threads) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, move_kernels(threads, false).scatter, threads, 0) !=
            cudaSuccess ||
        n < 1)
        n = 1024 / threads;
    return n;
}

cudaError_t launch_step(const Buffers& B, const Launch& L, cudaStream_t s, bool live) {
    const MoveKernels mk = move_kernels(L.threads_move, L.dense_move);
    cudaError_t e =
        launch_pdl(live ? mk.move_live : mk.move, live ? L.blocks_move_live : L.blocks_move, s, B, 0, L.threads_move);
    if (e == cudaSuccess && L.prefix_kernel) e = launch_pdl(k_tile_prefix, 1, s, B, 0, 1024);
    if (e == cudaSuccess) e = launch_pdl(k_scan, L.blocks_scan + 1 + kSortBlocks, s, B);
    if (e == cudaSuccess) e = launch_pdl(mk.scatter, L.blocks_scatter, s, B, 0, L.threads_move);
    if (e == cudaSuccess) e = launch_pdl(k_propose, L.blocks_propose, s, B, propose_smem(B));
    if (e == cudaSuccess) e = launch_pdl(k_accept, L.blocks_accept, s, B);
    return e;
}

// An event record that stays an event record when the stream is being
// captured into a graph (abm_profile_step replays the timed step as a graph).
static cudaError_t record_external(cudaEvent_t ev, cudaStream_t s) {
    return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
}

cudaError_t launch_step_timed(const Buffers& B, const Launch& L, cudaStream_t s, cudaEvent_t* ev, bool live) {
    const MoveKernels mk = move_kernels(L.threads_move, L.dense_move);
    record_external(ev[0], s);
    (live ? mk.move_live : mk.move)<<<live ? L.blocks_move_live : L.blocks_move, L.threads_move, 0, s>>>(B);
    record_external(ev[1], s);
    if (L.prefix_kernel) k_tile_prefix<<<1, 1024, 0, s>>>(B);
    record_external(ev[2], s);
    k_scan<<<L.blocks_scan + 1 + kSortBlocks, kThreads, 0, s>>>(B);
    record_external(ev[3], s);
    mk.scatter<<<L.blocks_scatter, L.threads_move, 0, s>>>(B);
    record_external(ev[4], s);
    k_propose<<<L.blocks_propose, kThreads, propose_smem(B), s>>>(B);
    record_external(ev[5], s);
    k_accept<<<L.blocks_accept, kThreads, 0, s>>>(B);
    record_external(ev[6], s);
    return cudaGetLastError();
}

cudaError_t prepare_kernels() { return cudaSuccess; }

cudaError_t launch_init(const Buffers& B, const Launch& L, cudaStream_t s, uint32_t sim, uint32_t base,
                        uint32_t n0, const uint32_t* d_species_end, uint32_t n_sp) {
    if (n0 == 0) return cudaSuccess;
    k_init<<<L.blocks_agents, kThreads, 0, s>>>(B, sim, base, n0, d_species_end, n_sp);
    return cudaGetLastError();
}

cudaError_t launch_observe(const Buffers& B, const Launch& L, cudaStream_t s, int32_t only_sim, int want_digest) {
    k_observe<<<L.blocks_agents, kThreads, 0, s>>>(B, only_sim, want_digest);
    return cudaGetLastError();
}

cudaError_t launch_compact(const Buffers& B, const Launch& L, cudaStream_t s) {
    k_compact<<<L.blocks_agents, kThreads, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_monitor(const Buffers& B, const Launch& L, cudaStream_t s, int32_t sim) {
    k_monitor_pass<<<L.blocks_agents, kThreads, 0, s>>>(B, (uint32_t)sim);
    k_monitor_eval<<<1, 1, 0, s>>>(B, (uint32_t)sim);
    return cudaGetLastError();
}

cudaError_t launch_dump(const Buffers& B, const Launch& L, cudaStream_t s, int32_t sim, void* d_out,
                        uint32_t cap) {
    uint4* lo = reinterpret_cast<uint4*>(d_out);
    uint2* hi = reinterpret_cast<uint2*>(lo + cap);
    k_dump<<<L.blocks_agents, kThreads, 0, s>>>(B, sim, lo, hi, cap);
    return cudaGetLastError();
}

// One simulation's counts vector (n words from src) and the control words,
// written by one block straight into a pinned host slot: the host sees them
// once an event recorded after this launch has completed.  One launch in
// stream order behind the step, where two copy-engine transfers would each
// wait for the step and hold the next one back.
__global__ void __launch_bounds__(kThreads) k_readout(const uint64_t* __restrict__ src, uint32_t n,
                                                      const Ctl* __restrict__ ctl, uint64_t* dst) {
    for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
    const uint32_t* c = reinterpret_cast<const uint32_t*>(ctl);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst + 512);
    for (uint32_t k = threadIdx.x; k < sizeof(Ctl) / 4; k += blockDim.x) d[k] = c[k];
    __threadfence_system();
}

cudaError_t launch_readout(const uint64_t* src, uint32_t n, const Ctl* ctl, uint64_t* dst, cudaStream_t s) {
    k_readout<<<1, kThreads, 0, s>>>(src, n, ctl, dst);
    return cudaGetLastError();
}

cudaError_t launch_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n,
                                cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_debug_philox<<<blocks, 256, 0, s>>>(reinterpret_cast<const uint4*>(ctr), reinterpret_cast<const uint2*>(key),
                                          reinterpret_cast<uint4*>(out), n);
    return cudaGetLastError();
}

}  // namespace abm
