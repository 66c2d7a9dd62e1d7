/*
 * abm.h — C ABI of the B300 molecule-agent step engine.
 *
 * The engine advances a 3D agent-based simulation in which every molecule is
 * an agent (paper, Sec. 2 "Materials and Methods": molecules are spheres that
 * diffuse, bind substrates or inhibitors by spatial proximity, release
 * products after a turnover time, are produced by expressors at a fixed rate
 * and move between compartments at translocation rates).  The inputs follow
 * the paper's list of what a model needs (Sec. 2, footnote 1): the simulated
 * volume, initial amounts, per-molecule properties (diffusion from molecular
 * size), reactions with partners, rates and products, compartment volumes
 * and translocation rates, and expression rates.
 *
 * One step of every simulation runs: first-order events (release of bound
 * complexes, conversion/degradation, expression), a Brownian move with
 * reflecting walls, rejecting spherical walls and membrane crossing, a cell
 * grid rebuilt by histogram / exclusive scan / scatter, a proximity proposal
 * over the cells a contact radius can reach (the 27-cell neighbourhood pruned
 * to the reachable cells), a nearest-partner handshake (atomicMin on a packed (dist^2, id)
 * key), reaction application and births.  All state is integer; all
 * randomness is Philox4x32-10 keyed by (seed, step, agent id), so a run is
 * bit-reproducible and independent of storage order.
 *
 * Conventions for every call:
 *  - Return value: an abm_status.  After any failure other than ABM_EINVAL
 *    at creation, the handle is in a failed state: every call except
 *    abm_*_last_error and abm_*_destroy returns ABM_ESTATE.
 *  - Host pointers are read during the call only (copied); the caller keeps
 *    ownership.  Device memory passed as `arena` and the `stream` belong to
 *    the caller and must outlive the handle.
 *  - abm_*_step only enqueues work on the stream and returns.  Errors found
 *    on the device (capacities exceeded, id space exhausted) are sticky and
 *    reported by the next synchronising call (counts, counts_finish, digest,
 *    dump, sync, monitor read).  No call waits on the device beyond a stream
 *    synchronisation.
 *  - Not thread-safe: one host thread per handle at a time.
 */
#ifndef ABM_H
#define ABM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ABM_OK = 0,
    ABM_EINVAL = -1,     /* invalid model or argument; nothing was created */
    ABM_ENOMEM = -2,     /* device allocation failed or arena too small    */
    ABM_ECUDA = -3,      /* a CUDA runtime call failed                     */
    ABM_ETIMEOUT = -4,   /* reserved: no call waits on the device today      */
    ABM_ECAPACITY = -5,  /* agents, cells, births or sims exceed capacity  */
    ABM_EDEVICE = -6,    /* no usable CUDA device (sm_103 required)        */
    ABM_ESTATE = -7      /* handle already failed, or bad sim index        */
} abm_status;

enum { ABM_CONVERT = 0, ABM_BIND = 1 };
enum { ABM_CUBE = 0, ABM_SPHERE = 1 };

/* A molecular species (paper Sec. 2: molecule classes and per-species
 * properties).  D_um2_s is the Stokes-Einstein diffusion coefficient the
 * caller derived from the molecular weight; 0 makes an immobile agent (gene
 * site).  An expressor is a species with p_emit > 0. */
typedef struct {
    uint32_t initial_count;  /* agents placed at creation                  */
    double   D_um2_s;        /* diffusion coefficient, um^2/s, >= 0        */
    int32_t  compartment;    /* compartment of the initial agents          */
    double   p_cross;        /* probability per attempted crossing, [0,1]  */
    double   p_uni;          /* first-order conversion per step, [0,1]     */
    int32_t  uni_to;         /* product of the conversion; -1 = death      */
    double   p_emit;         /* birth probability per step, [0,1]          */
    int32_t  emit_species;   /* species of the child; -1 = none            */
} abm_species;

/* A bimolecular reaction (paper Sec. 2: interacting partners, rates and
 * products).  Agent of species a proposes to agent of species b when they
 * are within radius_nm; CONVERT changes both at once, BIND forms a complex
 * that releases (prod_a, prod_b) with p_release per step (the turnover time).
 * Each unordered species pair has at most one reaction; a != b. */
typedef struct {
    int32_t a, b;
    int32_t kind;            /* ABM_CONVERT | ABM_BIND                     */
    int32_t prod_a, prod_b;  /* species afterwards; -1 = the agent dies    */
    double  radius_nm;       /* contact radius (> 0, <= the grid cell)     */
    double  p_bind;          /* Bernoulli per eligible contact, [0,1]      */
    double  p_release;       /* BIND only: per step, [0,1]                 */
} abm_reaction;

/* Compartment 0 is the root (a cube of edge size_um or a sphere of diameter
 * size_um).  Compartments 1..3 are spheres (diameter size_um) inside the
 * root, centred at the root centre plus center_um, not overlapping (the
 * nucleus of paper Sec. 3.4). */
typedef struct {
    int32_t shape;           /* ABM_CUBE (root only) | ABM_SPHERE          */
    double  size_um;
    int32_t parent;          /* -1 for the root, 0 for a child             */
    double  center_um[3];
} abm_compartment;

typedef struct {
    const abm_species*     species;       /* n_species in [1, 64]          */
    uint32_t               n_species;
    const abm_reaction*    reactions;     /* n_reactions in [0, 255]       */
    uint32_t               n_reactions;
    const abm_compartment* compartments;  /* n_compartments in [1, 4]      */
    uint32_t               n_compartments;
    double                 dt_s;          /* time step, > 0                */
    double                 unit_nm;       /* position quantum, > 0 (0.1)   */
} abm_model;
/* The root's edge (cube) or diameter (sphere), in units of unit_nm, must
 * lie in [2, 2^21): positions are stored in 21 bits per axis (209.7 um at
 * 0.1 nm).  Outside that range abm_create and abm_batch_add return
 * ABM_EINVAL. */

/* Options of a single simulation.  Zero-initialise and set what you need. */
typedef struct {
    uint64_t       capacity_agents;  /* 0 = initial count * 1.25 + 65536  */
    uint32_t       cell_log2;        /* grid cell = 2^k units; 0 = auto    */
    uint32_t       births_per_step;  /* births one step may add; 0 = 8192;
                                        clamped to the agent capacity      */
    void*          arena;            /* device memory, or NULL = library   */
    size_t         arena_bytes;
    void*          stream;           /* cudaStream_t, or NULL = library    */
    const int16_t* ncdf_table;       /* 65536 entries or NULL = built in   */
} abm_options;

/* Options of a batch of simulations stepped together. */
typedef struct {
    uint64_t       capacity_agents;  /* slots shared by all sims (> 0)     */
    uint64_t       capacity_cells;   /* grid cells shared by all sims      */
    uint32_t       max_sims;         /* 1..2048                            */
    uint32_t       births_per_step;  /* births one step may add to EACH
                                        simulation (its segment of the births
                                        buffer, 8 bytes per birth and slot);
                                        0 = 8192; clamped to capacity_agents */
    void*          arena;
    size_t         arena_bytes;
    void*          stream;
    const int16_t* ncdf_table;
    uint32_t       blocks_per_sm;    /* CTAs per SM for the move and scatter
                                        kernels (grid-stride); 0 = as many as fit
                                        on an SM at once */
    /* Launch shape (an autotuner's knobs; no choice changes a result): */
    uint32_t       threads_per_block;/* block size of the move and scatter
                                        kernels: 128, 256 or 512; 0 = 128
                                        for capacities from 2^20 to 2^21
                                        agents, else 256                     */
    uint32_t       propose_chunk;    /* sorted agents per block of the
                                        proximity search (a block covers
                                        several small simulations or part of a
                                        large one): 1024, 2048 or 4096;
                                        0 = by capacity                      */
} abm_batch_options;

/* Layout of abm_*_counts output (uint64 each):
 *   [n_species * n_compartments free agents, index species*n_comp + comp]
 *   [n_reactions bound complexes][next_id]
 * One dump record per agent (hidden partners of complexes included), sorted
 * by id, 24 bytes: */
typedef struct {
    uint32_t id;
    uint8_t  species, compartment;
    uint8_t  flags;          /* 1 carrier of a complex, 2 hidden, 4 reactant a */
    uint8_t  reaction;       /* 0xFF when free                             */
    int32_t  x, y, z;        /* units of unit_nm; hidden: carrier's place  */
    uint32_t partner;        /* 0xFFFFFFFF when free                       */
} abm_record;

/* ---------------- single simulation ---------------- */
typedef struct abm_sim abm_sim;

/* Bytes of device memory a simulation needs for these model and options
 * (the arena must be 256-byte aligned).  Returns 0 for an invalid model. */
size_t      abm_arena_bytes(const abm_model* model, const abm_options* opt);
abm_status  abm_create(const abm_model* model, uint64_t seed, const abm_options* opt,
                       abm_sim** out);
/* Grid of a model (host only, no device work): the cell edge 2^(*shift_out)
 * units chosen for cell_log2 (0 = automatic: about one agent per cell at the
 * initial density, never below the largest contact radius) and the number of
 * cells, for sizing a batch's capacity_cells.  ABM_EINVAL for invalid input. */
abm_status  abm_model_grid(const abm_model* model, uint32_t cell_log2, uint32_t* shift_out,
                           uint64_t* cells_out);
/* Resume a simulation from a checkpoint: the model and seed it was created
 * with, the records abm_dump returned (any order), and its step counter
 * (abm_step_index) and next id (last entry of abm_counts) at the time of the
 * dump.  All randomness is keyed by (seed, step, id), so continuing the
 * restored simulation reproduces the original trajectory bit for bit.
 * Records are checked (ids unique and below next_id, places inside the
 * domain and in their compartment, complexes complete): ABM_EINVAL
 * otherwise.  The model's initial counts are ignored. */
abm_status  abm_restore(const abm_model* model, uint64_t seed, const abm_options* opt,
                        const abm_record* records, size_t n_records, uint32_t step,
                        uint32_t next_id, abm_sim** out);
abm_status  abm_step(abm_sim* sim, uint32_t n);
abm_status  abm_counts(abm_sim* sim, uint64_t* out, size_t cap, size_t* n_out);
/* Pipelined counts of one simulation: see abm_batch_counts_begin below. */
abm_status  abm_counts_begin(abm_sim* sim, uint32_t slot);
abm_status  abm_counts_finish(abm_sim* sim, uint32_t slot, uint64_t* out, size_t cap, size_t* n_out);
abm_status  abm_live_counts(abm_sim* sim, int on);  /* see abm_batch_live_counts */
abm_status  abm_digest(abm_sim* sim, uint64_t* out);
abm_status  abm_dump(abm_sim* sim, abm_record* out, size_t cap, size_t* n_out);
abm_status  abm_sync(abm_sim* sim);
abm_status  abm_step_index(abm_sim* sim, uint32_t* out);
/* Number of grid cells of the simulation (host-side value, no device work). */
abm_status  abm_grid_cells(abm_sim* sim, uint64_t* out);
const char* abm_last_error(const abm_sim* sim);
void        abm_destroy(abm_sim* sim);        /* NULL-safe */

/* ---------------- batch of simulations ---------------- */
typedef struct abm_batch abm_batch;

size_t      abm_batch_arena_bytes(const abm_batch_options* opt);
abm_status  abm_batch_create(const abm_batch_options* opt, abm_batch** out);
/* Admit a simulation between steps: validates the model, places its agents
 * (on the device) and returns its slot in *sim_id.  cell_log2 as above.
 * Synchronises the stream.  ABM_ECAPACITY if agents, cells or slots run out. */
abm_status  abm_batch_add(abm_batch* b, const abm_model* model, uint64_t seed,
                          uint32_t cell_log2, int32_t* sim_id);
/* abm_restore into a batch slot (synchronises, like abm_batch_add). */
abm_status  abm_batch_restore(abm_batch* b, const abm_model* model, uint64_t seed,
                              uint32_t cell_log2, const abm_record* records, size_t n_records,
                              uint32_t step, uint32_t next_id, int32_t* sim_id);
/* Freeze a simulation once its step counter reaches max_step (absolute):
 * later steps keep its agents in place without advancing them, so a server
 * can step a batch in fixed epochs and still read every simulation at its
 * exact last step.  0xFFFFFFFF (the default) never freezes.  Synchronises. */
abm_status  abm_batch_set_max_step(abm_batch* b, int32_t sim_id, uint32_t max_step);
/* Retire a simulation: its agents are dropped by the next step's grid build
 * and its slot, agents and cells become free for later admissions. */
abm_status  abm_batch_remove(abm_batch* b, int32_t sim_id);
abm_status  abm_batch_step(abm_batch* b, uint32_t n);
abm_status  abm_batch_counts(abm_batch* b, int32_t sim_id, uint64_t* out, size_t cap,
                             size_t* n_out);
abm_status  abm_batch_digest(abm_batch* b, int32_t sim_id, uint64_t* out);
abm_status  abm_batch_dump(abm_batch* b, int32_t sim_id, abm_record* out, size_t cap,
                           size_t* n_out);
abm_status  abm_batch_sync(abm_batch* b);
/* Status of one simulation of the batch (synchronises).  A simulation whose
 * births in one step exceed births_per_step stops there (Sec. 2 and
 * Sec. 3.4: expression births): it is frozen at that step with a corrupt
 * state, this call and its counts, digest, dump and monitor reads return
 * ABM_ECAPACITY (message in abm_batch_last_error), and every other
 * simulation of the batch goes on unaffected; the caller removes it.  For a
 * handle of abm_create / abm_restore the same error fails the handle.
 * Exceeding the batch's agent capacity still fails the whole batch.
 * ABM_ESTATE for a free slot. */
abm_status  abm_batch_sim_status(abm_batch* b, int32_t sim_id);
/* Pipelined counts (the readout of Sec. 2, at every step if wanted, without
 * stalling the device): _begin queues the count pass for the state after the
 * steps issued so far and a one-block kernel that writes the counts into
 * pinned host slot `slot` (0 .. ABM_READ_SLOTS - 1), and returns at once; _finish waits for that slot and
 * writes the counts (layout as abm_batch_counts) to out[0..cap).  A caller
 * that steps, begins slot k % 2 and finishes slot (k - 1) % 2 keeps the
 * device busy while it reads.  ABM_EINVAL for a bad slot, _begin on a slot
 * that is not finished, _finish on one that was not begun, or cap below the
 * count; device errors surface at _finish as in abm_batch_counts. */
#define ABM_READ_SLOTS 4
abm_status  abm_batch_counts_begin(abm_batch* b, int32_t sim_id, uint32_t slot);
/* Live counts (on = 1): every step also leaves the counts of its result in a
 * device buffer; the move pass counts the moved agents as it writes them, the
 * acceptance walk and the births add their changes.  abm_batch_counts_begin
 * then only copies them, with no pass over the agents, whenever a step has
 * run since live counts were switched on and since the last admission,
 * restore or removal; otherwise it counts as before.  The values are the same
 * either way.  Costs one shared-memory add per agent per step while on.
 * Asynchronous; on = 0 switches it off. */
abm_status  abm_batch_live_counts(abm_batch* b, int on);
abm_status  abm_batch_counts_finish(abm_batch* b, uint32_t slot, uint64_t* out, size_t cap,
                                    size_t* n_out);
abm_status  abm_batch_live_agents(abm_batch* b, uint64_t* out);  /* syncs */
const char* abm_batch_last_error(const abm_batch* b);
void        abm_batch_destroy(abm_batch* b);  /* NULL-safe */

/* ---------------- threshold monitor ---------------- */
/* Sec. 2 (simulator description): the user designates molecular species
 * to follow continuously and sets a concentration threshold for a time
 * window; the simulator then classifies the cell from whether the level
 * passes it (the paper's ppERK example: above the healthy level early means
 * aberrant signalling, and a drug that brings it back below means a return to
 * normal).  Here a monitor watches one simulation:
 *
 *   value(t) = sum_k weights[k] * counts[k](t)
 *
 * over the counts layout above (free agents by species and compartment,
 * bound complexes by reaction), at the state after t completed steps, for
 * every t in [step_begin, step_end) with (t - step_begin) % period == 0.  A
 * state passes when value > threshold (above = 1) or value < threshold
 * (above = 0).  Each due state is evaluated exactly once: by the step that
 * starts from it (the sum is taken inside that step's move kernel, so a
 * monitor costs one weight lookup per agent and no extra pass over memory),
 * or, for the state no step has started from yet, by abm_*_monitor_read.
 * Results are exact integers and do not depend on when reads happen. */
typedef struct {
    uint32_t step_begin;     /* first step of the window                      */
    uint32_t step_end;       /* one past the last; 0xFFFFFFFF = open-ended    */
    uint32_t period;         /* >= 1                                          */
    int32_t  above;          /* 1: passes when value > threshold, 0: < ...    */
    int64_t  threshold;
} abm_monitor;

typedef struct {
    int64_t  value;          /* value at the last evaluation                  */
    uint32_t last_step;      /* step of the last evaluation                   */
    uint32_t first_pass;     /* first evaluated step that passed, 0xFFFFFFFF = none */
    uint32_t n_evaluated;
    uint32_t n_passed;
    int32_t  state;          /* last evaluation: 1 passed, 0 not, -1 none yet */
    uint32_t reserved;
} abm_monitor_state;

/* Install (or replace, resetting its state) the monitor of a simulation.
 * weights: n_weights <= counts length - 1 entries (the next-id entry is not a
 * count), the rest taken as 0, each in [-2^20, 2^20].  ABM_EINVAL for bad
 * weights, period 0 or step_end <= step_begin; ABM_ESTATE for a free slot.
 * Synchronises.  Removing a simulation clears its monitor. */
abm_status  abm_batch_monitor_set(abm_batch* b, int32_t sim_id, const abm_monitor* m,
                                  const int32_t* weights, size_t n_weights);
abm_status  abm_batch_monitor_clear(abm_batch* b, int32_t sim_id);   /* synchronises */
/* State of the monitor after evaluating the current state if it is due,
 * and the last min(n_evaluated, 1024) evaluated values, oldest first, in
 * trace[0..cap) (*n_out = how many there are).  ABM_ESTATE without a
 * monitor.  Synchronises. */
abm_status  abm_batch_monitor_read(abm_batch* b, int32_t sim_id, abm_monitor_state* out,
                                   int64_t* trace, size_t cap, size_t* n_out);
abm_status  abm_monitor_set(abm_sim* sim, const abm_monitor* m, const int32_t* weights,
                            size_t n_weights);
abm_status  abm_monitor_clear(abm_sim* sim);
abm_status  abm_monitor_read(abm_sim* sim, abm_monitor_state* out, int64_t* trace, size_t cap,
                             size_t* n_out);

/* ---------------- dump without allocation ---------------- */
/* The same id-sorted records as abm_dump, for callers that cannot allocate
 * device memory at the time of the call: abm_dump allocates a device staging
 * buffer per call (cudaMalloc, which also synchronises the device), which a
 * per-step monitor hook with a time budget, or a host application whose own
 * allocator owns all device memory, cannot allow.  This call allocates
 * nothing: records are staged in a fixed device array of 131,072 records
 * (3 MiB) that every GPU loading the library holds until exit, then copied
 * into `out` (host, cap records) and sorted there in place.  The paper has no
 * counterpart; it is a property of this library only.
 *  - out == NULL: returns the record count in *n_out (a size query).
 *  - More than 131,072 records: ABM_ECAPACITY, with the limit named in
 *    abm_last_error; the handle stays usable (use abm_dump instead).
 *  - cap below the record count: ABM_EINVAL (message in abm_last_error);
 *    the handle stays usable.
 *  - Call it with the device that was current when the handle was created
 *    (the array is per device); with another device current it returns
 *    ABM_EDEVICE and changes nothing.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - A failing CUDA call inside it returns ABM_ECUDA and leaves the handle
 *    destroy-only, like any other call.
 *  - All calls share the array (each clears its counter first); calls that
 *    overlap on the GPU race.  Synchronous. */
abm_status  abm_dump_noalloc(abm_sim* sim, abm_record* out, size_t cap, size_t* n_out);

/* ---------------- profiling ---------------- */
/* Runs n steps with a CUDA event on the stream before and after each of the
 * step's kernels (the kernels launched one after another, without the
 * step's overlap between consecutive kernels; the launches and events are
 * replayed as one CUDA graph, captured on first use, so that host launch
 * latency falls outside the timed intervals), and writes the summed time of
 * each kernel in milliseconds to kernel_ms[0..5] (n_kernels >= 6; names from
 * abm_kernel_name; slot 1, k_tile_prefix, runs only on grids of more than
 * 8192 tiles of 8192 cells and reads 0 otherwise).  Synchronous.  The state
 * advances exactly as abm_step. */
abm_status  abm_profile_step(abm_sim* sim, uint32_t n, float* kernel_ms, uint32_t n_kernels);
abm_status  abm_batch_profile_step(abm_batch* b, uint32_t n, float* kernel_ms, uint32_t n_kernels);
/* Name of step kernel k (0..5), or NULL. */
const char* abm_kernel_name(uint32_t k);

/* ---------------- building blocks (host or debug) ---------------- */
/* The Gaussian inverse-CDF table the engine uses when none is given:
 * Z[i] = round(4096 * inv_Phi((i + 1/2) / 65536)), host computation. */
void        abm_ncdf_table(int16_t* out65536);
/* Runs the engine's device Philox4x32-10 on n (counter, key) pairs given as
 * host arrays ctr[4n], key[2n]; writes out[4n] (host).  Synchronous. */
abm_status  abm_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                             size_t n);
/* Testing hook (host-side failure injection; no counterpart in the paper):
 * the next abm_step / abm_batch_step call in this process reports
 * `cuda_error` (a cudaError_t value, nonzero) as the result of its launch
 * without launching anything, so the call returns ABM_ECUDA and the handle
 * becomes destroy-only (ABM_ESTATE), exactly as after a real launch failure.
 * The device and other handles are unaffected.  0 clears a pending injection. */
void        abm_debug_inject_launch_error(int cuda_error);
/* Library version string. */
const char* abm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ABM_H */
