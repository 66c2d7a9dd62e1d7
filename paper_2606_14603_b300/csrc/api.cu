// api.cu — host side of the C ABI (include/abm.h): model validation and
// compilation to integers, arena layout, admission of simulations into a
// batch, CUDA-graph capture of the step, and the observation calls.
//
// Physical-to-integer conversions follow one rule: evaluate left to right in
// IEEE double, round half away from zero (llround).
//   extent      cube: llround(edge_um * 1000 / unit_nm); sphere: 2 r with
//               r = llround(diameter_um * 1000 / unit_nm / 2)
//   M           llround(sqrt(2 D dt) * 1000 / unit_nm * 2^20)
//   thresholds  floor(p * 2^32)
//   radius      llround(radius_nm / unit_nm)
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/abm.h"
#include "engine.cuh"

using namespace abm;

namespace {

constexpr int kTile = kScanTile;
constexpr size_t kAlign = 256;

// ------------------------------------------------------------------------
// Built-in Gaussian table.  inv_Phi on the lower half by Newton's method on
// Phi(x) - p (Phi from erfc), started from the rational approximation of
// Abramowitz & Stegun 26.2.23; the upper half mirrors it.
double normal_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

double inv_normal_lower(double p) {
    const double t = std::sqrt(-2.0 * std::log(p));
    double x = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                         (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
    for (int it = 0; it < 100; it++) {
        const double dens = std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI);
        const double step = (normal_cdf(x) - p) / dens;
        x -= step;
        if (std::fabs(step) <= 1e-16 * std::fabs(x)) break;
    }
    return x;
}

void build_table(int16_t* out) {
    for (int i = 0; i < 32768; i++) {
        const double q = inv_normal_lower((i + 0.5) / 65536.0);
        const int16_t mag = (int16_t)std::floor(-4096.0 * q + 0.5);
        out[i] = (int16_t)-mag;
        out[65535 - i] = mag;
    }
}

// The default table, built once per process (about 13 ms of host work).
const int16_t* default_table() {
    static std::vector<int16_t> table;
    static std::once_flag once;
    std::call_once(once, [] {
        table.resize(65536);
        build_table(table.data());
    });
    return table.data();
}

uint64_t threshold(double p) { return (uint64_t)std::floor(p * 4294967296.0); }
bool prob_ok(double p) { return std::isfinite(p) && p >= 0.0 && p <= 1.0; }

// ------------------------------------------------------------------------
struct Compiled {
    ModelDev dev;
    SimDev geo;  // geometry part of the sim entry
    int64_t Rmax = 0;
    uint64_t n0 = 0;
    uint32_t species_end[kMaxSpecies] = {};
    double volume = 0;  // root volume in units^3
};

abm_status compile_model(const abm_model* m, Compiled* c, std::string* err) {
    auto bad = [&](const char* msg) {
        *err = msg;
        return ABM_EINVAL;
    };
    if (!m) return bad("model is NULL");
    if (!m->species || m->n_species < 1 || m->n_species > (uint32_t)kMaxSpecies)
        return bad("n_species must be in [1, 64]");
    if (m->n_reactions > (uint32_t)kMaxReactions || (m->n_reactions && !m->reactions))
        return bad("n_reactions must be in [0, 255]");
    if (!m->compartments || m->n_compartments < 1 || m->n_compartments > (uint32_t)kMaxComp)
        return bad("n_compartments must be in [1, 4]");
    const double dt = m->dt_s, unit = m->unit_nm;
    if (!(std::isfinite(dt) && dt > 0) || !(std::isfinite(unit) && unit > 0))
        return bad("dt_s and unit_nm must be positive");
    std::memset(&c->dev, 0, sizeof(c->dev));
    std::memset(&c->geo, 0, sizeof(c->geo));
    std::memset(c->dev.rx_of, 0xFF, sizeof(c->dev.rx_of));
    const uint32_t n_sp = m->n_species, n_rx = m->n_reactions, n_comp = m->n_compartments;

    // geometry
    const abm_compartment* cm = m->compartments;
    if (cm[0].parent != -1) return bad("compartment 0 must be the root (parent -1)");
    if (!(std::isfinite(cm[0].size_um) && cm[0].size_um > 0)) return bad("root size must be positive");
    int64_t ext;
    SimDev& g = c->geo;
    if (cm[0].shape == ABM_CUBE) {
        ext = llround(cm[0].size_um * 1000.0 / unit);
        g.root_sphere = 0;
        g.c0[0] = g.c0[1] = g.c0[2] = (int32_t)(ext / 2);
        c->volume = (double)ext * ext * ext;
    } else if (cm[0].shape == ABM_SPHERE) {
        const int64_t r = llround(cm[0].size_um * 1000.0 / unit / 2.0);
        ext = 2 * r;
        g.root_sphere = 1;
        g.root_r2 = r * r;
        g.c0[0] = g.c0[1] = g.c0[2] = (int32_t)r;
        c->volume = 4.0 / 3.0 * M_PI * (double)r * r * r;
    } else {
        return bad("unknown root shape");
    }
    if (ext < 2 || ext >= kPosLimit) return bad("root extent must be in [2, 2^21) position units");
    g.ext = (int32_t)ext;
    g.n_comp = (int32_t)n_comp;
    for (uint32_t k = 1; k < n_comp; k++) {
        if (cm[k].parent != 0 || cm[k].shape != ABM_SPHERE) return bad("compartments 1..3 must be spheres in the root");
        if (!(std::isfinite(cm[k].size_um) && cm[k].size_um > 0)) return bad("compartment size must be positive");
        const int64_t r = llround(cm[k].size_um * 1000.0 / unit / 2.0);
        if (r < 1) return bad("child sphere too small");
        int64_t cc[3];
        for (int d = 0; d < 3; d++) {
            if (!std::isfinite(cm[k].center_um[d])) return bad("bad compartment centre");
            cc[d] = g.c0[d] + llround(cm[k].center_um[d] * 1000.0 / unit);
            g.cc[k][d] = (int32_t)cc[d];
        }
        g.cr2[k] = r * r;
        if (g.root_sphere) {
            const int64_t room = ext / 2 - r;
            int64_t d2 = 0;
            for (int d = 0; d < 3; d++) d2 += (cc[d] - g.c0[d]) * (cc[d] - g.c0[d]);
            if (room < 0 || d2 > room * room) return bad("child sphere leaves the root");
        } else {
            for (int d = 0; d < 3; d++)
                if (cc[d] - r < 0 || cc[d] + r > ext) return bad("child sphere leaves the root");
        }
        for (uint32_t j = 1; j < k; j++) {
            const int64_t rj = (int64_t)llround(std::sqrt((double)g.cr2[j]));
            int64_t d2 = 0;
            for (int d = 0; d < 3; d++) d2 += (cc[d] - g.cc[j][d]) * (int64_t)(cc[d] - g.cc[j][d]);
            if (d2 <= (r + rj) * (r + rj)) return bad("child spheres overlap");
        }
    }

    // bound on |Z| for any int16 table, so that one fold always suffices
    const int zmax = 32768;
    uint64_t total = 0;
    for (uint32_t i = 0; i < n_sp; i++) {
        const abm_species& s = m->species[i];
        if (!(std::isfinite(s.D_um2_s) && s.D_um2_s >= 0)) return bad("diffusion coefficient must be >= 0");
        if (!prob_ok(s.p_cross) || !prob_ok(s.p_uni) || !prob_ok(s.p_emit)) return bad("species probability outside [0,1]");
        if (s.compartment < 0 || s.compartment >= (int32_t)n_comp) return bad("species compartment out of range");
        if (s.uni_to < -1 || s.uni_to >= (int32_t)n_sp) return bad("uni_to names an unknown species");
        if (s.emit_species < -1 || s.emit_species >= (int32_t)n_sp) return bad("emit_species names an unknown species");
        SpeciesDev& d = c->dev.sp[i];
        const double sigma_delta = std::sqrt(2.0 * s.D_um2_s * dt) * 1000.0 / unit;
        const long long M = llround(sigma_delta * 1048576.0);
        if (M < 0 || M >= (1ll << 32)) return bad("diffusion step too large for the time step");
        if ((((uint64_t)zmax * (uint64_t)M + 0x80000000ull) >> 32) > (uint64_t)ext)
            return bad("diffusion step exceeds the domain");
        d.M = (uint32_t)M;
        d.thr_uni = threshold(s.p_uni);
        d.thr_emit = s.emit_species >= 0 ? threshold(s.p_emit) : 0;
        d.thr_cross = threshold(s.p_cross);
        d.uni_to = (int16_t)s.uni_to;
        d.emit = (int16_t)s.emit_species;
        d.has_event = (d.thr_uni || d.thr_emit) ? 1 : 0;
        d.init_comp = (uint16_t)s.compartment;
        total += s.initial_count;
        c->species_end[i] = (uint32_t)std::min<uint64_t>(total, 0xFFFFFFFFull);
    }
    if (total >= 0xFFFFFFF0ull) return bad("too many agents for 32-bit ids");
    c->n0 = total;
    for (uint32_t r = 0; r < n_rx; r++) {
        const abm_reaction& q = m->reactions[r];
        if (q.a < 0 || q.a >= (int32_t)n_sp || q.b < 0 || q.b >= (int32_t)n_sp) return bad("reaction names an unknown species");
        if (q.a == q.b) return bad("A + A reactions are not supported");
        if (q.kind != ABM_CONVERT && q.kind != ABM_BIND) return bad("unknown reaction kind");
        if (q.prod_a < -1 || q.prod_a >= (int32_t)n_sp || q.prod_b < -1 || q.prod_b >= (int32_t)n_sp)
            return bad("reaction product names an unknown species");
        if (!prob_ok(q.p_bind) || !prob_ok(q.p_release)) return bad("reaction probability outside [0,1]");
        if (!std::isfinite(q.radius_nm)) return bad("reaction radius must be finite");
        if (c->dev.rx_of[q.a][q.b] != 0xFF || c->dev.rx_of[q.b][q.a] != 0xFF)
            return bad("two reactions for the same species pair");
        const long long R = llround(q.radius_nm / unit);
        if (R < 1 || R > 30000) return bad("reaction radius must be in [1, 30000] units");
        ReactionDev& d = c->dev.rx[r];
        d.thr_bind = threshold(q.p_bind);
        d.thr_rel = threshold(q.p_release);
        d.R = (int32_t)R;
        d.R2 = (uint32_t)(R * R);
        d.prod_a = (int16_t)q.prod_a;
        d.prod_b = (int16_t)q.prod_b;
        d.kind = (uint8_t)q.kind;
        d.carrier_a = !(m->species[q.b].D_um2_s < m->species[q.a].D_um2_s);
        d.a = (uint8_t)q.a;
        d.b = (uint8_t)q.b;
        c->dev.rx_of[q.a][q.b] = (uint8_t)r;
        c->dev.sp[q.a].partner_mask |= 1ull << q.b;
        c->dev.sp[q.a].rmax = std::max<int32_t>(c->dev.sp[q.a].rmax, (int32_t)R);
        c->Rmax = std::max<int64_t>(c->Rmax, R);
    }
    c->dev.n_sp = n_sp;
    c->dev.n_rx = n_rx;
    c->dev.n_comp = n_comp;
    c->dev.n_counts = n_sp * n_comp + n_rx + 1;
    return ABM_OK;
}

// Grid cell edge 2^shift: about one agent per cell at the initial density,
// never below the largest contact radius.
uint32_t auto_shift(const Compiled& c) {
    const double n = std::max<double>(1.0, (double)c.n0);
    const double h = std::cbrt(c.volume / n);
    int s = (int)std::floor(std::log2(std::max(h, 1.0)) + 0.5);
    int smin = 0;
    while ((1ll << smin) < c.Rmax) smin++;
    // at most 1024 cells per axis
    while ((c.geo.ext >> s) + 1 > 1024) s++;
    return (uint32_t)std::max(s, smin);
}

uint64_t cells_for(const Compiled& c, uint32_t shift) {
    const uint64_t gx = (uint64_t)(c.geo.ext >> shift) + 1;
    return gx * gx * gx;
}

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Births per step of one simulation (its segment of the births buffer):
// the option, or kDefaultBirths, at most the agent capacity (a step adds at
// most one child per agent), rounded up to even (16-byte segments).
uint32_t births_quota(uint64_t want, uint64_t cap_agents) {
    uint64_t q = want ? want : kDefaultBirths;
    q = std::min<uint64_t>(q, std::max<uint64_t>(cap_agents, 1));
    return (uint32_t)((q + 1) & ~1ull);
}

struct Layout {
    size_t off[48];
    size_t total;
};

// Sub-buffer sizes of a batch arena, in the order carved by carve().
Layout layout_for(uint64_t C, uint64_t K, uint32_t S, uint32_t Bc) {
    const uint64_t E = C / 2 + 1;
    const uint64_t Kpad = (K + kTile - 1) / kTile * kTile;
    const uint64_t tiles = Kpad / kTile + 1;
    const size_t sizes[] = {
        16 * C, 16 * C,                        // pm[2] (packed records with ids)
        4 * C, 4 * C,                          // apar[2]
        4 * C, 8 * C, 8 * C, (size_t)C,        // rk, acc, props, pflag
        16 * E, 4 * E,                         // extras: records, ranks
        8 * (size_t)Bc * S, 4 * ((size_t)S + 1),  // births: one segment per simulation slot, prefixes
        4 * (size_t)Bc * S, 4 * ((size_t)S + 1),  // sorted tiles of long births segments, their prefixes
        4 * Kpad, 4 * (Kpad + 8),              // cnt, start
        4 * kTileStride * tiles,               // tile counts (one per 128-byte line)
        4 * tiles,                             // tile prefixes
        sizeof(SimDev) * S, sizeof(ModelDev) * S,
        8 * (size_t)S * 512, 8 * (size_t)S,    // counts, digests
        2 * 8 * (size_t)S * 512,               // live counts, by step parity
        sizeof(MonDev) * S, 4 * (size_t)S * 512,   // threshold monitors, their weights
        8 * (size_t)S, 8 * (size_t)S * kMonTrace,  // monitor sums, evaluated values
        2 * 65536,                             // Gaussian table
        sizeof(Ctl),
        4 * kMaxSpecies,                       // staging for admissions
    };
    Layout L{};
    size_t o = 0;
    constexpr int n = (int)(sizeof(sizes) / sizeof(sizes[0]));
    static_assert(n < (int)(sizeof(L.off) / sizeof(L.off[0])), "layout table too small");
    for (int i = 0; i < n; i++) {
        L.off[i] = o;
        o += align_up(sizes[i]);
    }
    L.off[n] = o;
    L.total = o;
    return L;
}

}  // namespace

// ------------------------------------------------------------------------
struct abm_batch {
    int device = 0;                      // CUDA device current at creation (owns arena and stream)
    uint64_t cap_agents = 0, cap_cells = 0;
    uint32_t max_sims = 0, bquota = 0;
    bool single = false;                 // created by abm_create / abm_restore: a simulation's error fails the handle
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    bool own_arena = false;
    Buffers B{};
    Launch L{};
    uint32_t* staging = nullptr;
    Ctl* h_ctl = nullptr;                // pinned host copies: control block ...
    uint64_t* h_counts = nullptr;        // ... and one simulation's counts (512 words)
    struct ReadSlot {                    // pipelined counts reads
        uint64_t* host = nullptr;        // pinned: 512 counts, then a copy of the control block
        uint64_t* dev = nullptr;         // the same memory as the device addresses it
        cudaEvent_t done = nullptr;
        uint32_t n = 0;
        int32_t sim = -1;
        bool pending = false;
    };
    ReadSlot rs[ABM_READ_SLOTS];
    uint32_t epoch_host = 1;             // device epoch after the steps issued so far
    uint32_t live_on = 0;                // host copy of ctl.live_counts (source of its upload)
    bool live_valid = false;             // live counts hold the current state (a step ran with them on)
    cudaGraphExec_t g1 = nullptr, g8 = nullptr;
    cudaGraphExec_t g1_live = nullptr, g8_live = nullptr;  // the same with live counts, captured on first use
    // abm_profile_step: one step's kernels with an event before and after each,
    // as a graph (so that no host launch gap falls between an event and its
    // kernel), captured on first use, without and with live counts
    cudaGraphExec_t gprof[2] = {nullptr, nullptr};
    cudaEvent_t prof_ev[kStepKernels + 1] = {};
    uint32_t sim_errs_seen = 0;          // per-simulation errors already read from the device
    struct HostSim {
        int state = 0;  // 0 free, 1 active, 2 draining (removed, not yet stepped)
        abm_status status = ABM_OK;     // a per-simulation error read from the device (sticky)
        std::string err;
        uint32_t model_slot = 0;
        uint64_t n_cells = 0;
        uint32_t n_counts = 0;
        uint32_t shift = 0;
        bool monitor = false;
    };
    std::vector<HostSim> sims;
    std::vector<uint32_t> cell_off_host;  // persistent sources of async copies
    uint32_t n_cells_host = 0;
    uint32_t max_step_host = 0;
    std::vector<ModelDev> model_host;   // copies of the uploaded model tables
    std::vector<int> model_refs;
    uint32_t n_sims_used = 0;
    uint32_t n_monitors = 0;             // host copy of ctl.n_monitors (source of its upload)
    MonDev mon_host{};                   // source of a monitor upload
    std::vector<int32_t> mon_w_host;     // source of a weights upload
    bool failed = false;
    std::string err;
};

struct abm_sim {
    abm_batch* b = nullptr;
    int32_t id = -1;
};

namespace {

abm_status fail(abm_batch* b, abm_status st, const std::string& msg) {
    b->failed = true;
    b->err = msg;
    return st;
}

abm_status cuda_fail(abm_batch* b, cudaError_t e, const char* where) {
    return fail(b, ABM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Host-side failure injection for tests: the next step call reports this
// CUDA error as the result of its launch, without launching anything.
std::atomic<int> g_inject_launch_error{0};

#define CU(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(b, e_, #call); \
    } while (0)

abm_status check_device(std::string* msg) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        *msg = "no CUDA device";
        return ABM_EDEVICE;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
        *msg = "cannot query the CUDA device";
        return ABM_EDEVICE;
    }
    if (p.major != 10 || p.minor != 3) {
        char buf[128];
        std::snprintf(buf, sizeof buf, "device is sm_%d%d; this library is built for sm_103a", p.major, p.minor);
        *msg = buf;
        return ABM_EDEVICE;
    }
    return ABM_OK;
}

// Per-simulation errors (births of one step beyond a simulation's limit):
// read the error words of the simulations when the device has counted new
// ones; each failed simulation keeps its status, the batch goes on.  A
// handle created as a single simulation fails as a whole.
abm_status check_sim_errors(abm_batch* b, const Ctl& h) {
    if (h.sim_errs == b->sim_errs_seen) return ABM_OK;
    b->sim_errs_seen = h.sim_errs;
    std::vector<SimDev> sd(b->n_sims_used);
    if (!sd.empty()) {
        cudaError_t e = cudaMemcpyAsync(sd.data(), b->B.sims, sizeof(SimDev) * sd.size(), cudaMemcpyDeviceToHost,
                                        b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_fail(b, e, "reading simulation errors");
    }
    std::string first;
    for (uint32_t s = 0; s < b->n_sims_used; s++) {
        auto& hs = b->sims[s];
        if (!sd[s].err || hs.status != ABM_OK || hs.state == 0) continue;
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "simulation %u: births of one step exceed its limit of %u (birth %u); the simulation "
                      "is stopped, the other simulations go on", s, b->bquota, sd[s].err_info);
        hs.status = ABM_ECAPACITY;
        hs.err = buf;
        if (first.empty()) first = buf;
    }
    if (b->single && !first.empty()) return fail(b, ABM_ECAPACITY, first);
    return ABM_OK;
}

// Map the sticky device error word to a status.
abm_status check_ctl(abm_batch* b, const Ctl& h) {
    if (h.err == ERR_NONE) return check_sim_errors(b, h);
    char buf[160];
    abm_status st = ABM_ECAPACITY;
    const char* what = "capacity exceeded";
    switch (h.err) {
        case ERR_CAPACITY_AGENTS: what = "agent capacity exceeded"; break;
        case ERR_CAPACITY_EXTRAS: what = "release buffer capacity exceeded"; break;
        case ERR_CAPACITY_BIRTHS: what = "births per step exceed the limit"; break;
        case ERR_PLACEMENT: what = "could not place an agent in its compartment"; st = ABM_EINVAL; break;
        case ERR_ID_SPACE: what = "agent id space exhausted"; break;
        default: what = "device error"; st = ABM_ECUDA; break;
    }
    std::snprintf(buf, sizeof buf, "%s (code %u, info %u)", what, h.err, h.err_info);
    return fail(b, st, buf);
}

abm_status sync_and_check(abm_batch* b, Ctl* out_ctl = nullptr) {
    if (b->failed) return ABM_ESTATE;
    CU(cudaMemcpyAsync(b->h_ctl, b->B.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    const Ctl h = *b->h_ctl;
    if (out_ctl) *out_ctl = h;
    return check_ctl(b, h);
}

// The status of a simulation whose per-simulation error has been read
// (ABM_OK otherwise); its message goes to the batch's last error.
abm_status sim_status(abm_batch* b, int32_t sim) {
    const auto& hs = b->sims[sim];
    if (hs.status == ABM_OK) return ABM_OK;
    b->err = hs.err;
    return hs.status;
}

abm_status capture(abm_batch* b, bool live = false) {
    cudaStream_t cs;
    CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    for (int k = 0; k < 2; k++) {
        const int steps = k == 0 ? 1 : 8;
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            return cuda_fail(b, e, "cudaStreamBeginCapture");
        }
        for (int s = 0; s < steps; s++) launch_step(b->B, b->L, cs, live);
        e = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            return cuda_fail(b, e, "cudaStreamEndCapture");
        }
        cudaGraphExec_t* exec = live ? (k == 0 ? &b->g1_live : &b->g8_live) : (k == 0 ? &b->g1 : &b->g8);
        e = cudaGraphInstantiate(exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            return cuda_fail(b, e, "cudaGraphInstantiate");
        }
    }
    cudaStreamDestroy(cs);
    return ABM_OK;
}

// Re-pack every active simulation's cell range (keys are recomputed from
// positions every step, so offsets may change between steps).
abm_status repack_cells(abm_batch* b) {
    uint64_t off = 0;
    for (uint32_t s = 0; s < b->n_sims_used; s++) {
        auto& h = b->sims[s];
        if (h.state != 1) continue;
        b->cell_off_host[s] = (uint32_t)off;
        CU(cudaMemcpyAsync(&b->B.sims[s].cell_off, &b->cell_off_host[s], 4, cudaMemcpyHostToDevice, b->stream));
        off += h.n_cells;
    }
    b->n_cells_host = (uint32_t)off;
    CU(cudaMemcpyAsync(&b->B.ctl->n_cells, &b->n_cells_host, 4, cudaMemcpyHostToDevice, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return ABM_OK;
}

uint64_t cells_in_use(const abm_batch* b) {
    uint64_t off = 0;
    for (uint32_t s = 0; s < b->n_sims_used; s++)
        if (b->sims[s].state == 1) off += b->sims[s].n_cells;
    return off;
}

// Drop the agents of retired simulations (between steps) and free their slots.
abm_status compact(abm_batch* b, Ctl* h) {
    CU(cudaMemsetAsync(&b->B.ctl->n_compact, 0, 4, b->stream));
    CU(launch_compact(b->B, b->L, b->stream));
    uint32_t kept = 0;
    CU(cudaMemcpyAsync(&kept, &b->B.ctl->n_compact, 4, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    const uint32_t nxt = h->cur ^ 1u;
    CU(cudaMemcpyAsync(&b->B.ctl->cur, &nxt, 4, cudaMemcpyHostToDevice, b->stream));
    CU(cudaMemcpyAsync(&b->B.ctl->n_buf[nxt], &kept, 4, cudaMemcpyHostToDevice, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    for (auto& s : b->sims)
        if (s.state == 2) s.state = 0;
    h->cur = nxt;
    h->n_buf[nxt] = kept;
    return ABM_OK;
}

}  // namespace

// ------------------------------------------------------------------------
extern "C" {

const char* abm_version(void) { return "abm-b300 1.0 (sm_103a)"; }

void abm_ncdf_table(int16_t* out) {
    if (out) std::memcpy(out, default_table(), 2 * 65536);
}

size_t abm_batch_arena_bytes(const abm_batch_options* o) {
    if (!o || !o->capacity_agents || !o->capacity_cells || !o->max_sims || o->max_sims > (uint32_t)kMaxSims)
        return 0;
    const uint32_t births = births_quota(o->births_per_step, o->capacity_agents);
    return layout_for(o->capacity_agents, o->capacity_cells, o->max_sims, births).total;
}

abm_status abm_batch_create(const abm_batch_options* o, abm_batch** out) {
    if (!out) return ABM_EINVAL;
    *out = nullptr;
    if (!o || !o->capacity_agents || !o->capacity_cells || !o->max_sims || o->max_sims > (uint32_t)kMaxSims)
        return ABM_EINVAL;
    if (o->capacity_agents >= 0x7FFFFFFFull || o->capacity_cells >= 0xFFFFF000ull) return ABM_EINVAL;
    if (o->blocks_per_sm > 64) return ABM_EINVAL;
    if (o->threads_per_block && !valid_move_threads((int)o->threads_per_block)) return ABM_EINVAL;
    if (o->propose_chunk && o->propose_chunk != 1024 && o->propose_chunk != 2048 && o->propose_chunk != 4096)
        return ABM_EINVAL;
    const uint32_t births = births_quota(o->births_per_step, o->capacity_agents);
    std::string msg;
    abm_status st = check_device(&msg);
    if (st != ABM_OK) return st;
    abm_batch* b = new (std::nothrow) abm_batch();
    if (!b) return ABM_ENOMEM;
    b->cap_agents = o->capacity_agents;
    b->cap_cells = o->capacity_cells;
    b->max_sims = o->max_sims;
    b->bquota = births;
    const Layout lay = layout_for(b->cap_agents, b->cap_cells, b->max_sims, births);
    auto destroy_and = [&](abm_status s) {
        abm_batch_destroy(b);
        return s;
    };
    if (o->arena) {
        if (o->arena_bytes < lay.total || ((uintptr_t)o->arena % kAlign)) return destroy_and(ABM_ENOMEM);
        b->arena = (char*)o->arena;
        b->arena_bytes = o->arena_bytes;
    } else {
        if (cudaMalloc((void**)&b->arena, lay.total) != cudaSuccess) {
            cudaGetLastError();
            b->arena = nullptr;
            return destroy_and(ABM_ENOMEM);
        }
        b->own_arena = true;
        b->arena_bytes = lay.total;
    }
    if (o->stream) {
        b->stream = (cudaStream_t)o->stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return destroy_and(ABM_ECUDA);
        b->own_stream = true;
    }
    if (cudaMallocHost((void**)&b->h_ctl, sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_counts, 8 * 512) != cudaSuccess) {
        cudaGetLastError();
        return destroy_and(ABM_ENOMEM);
    }
    for (auto& r : b->rs)
        if (cudaMallocHost((void**)&r.host, 8 * 512 + sizeof(Ctl)) != cudaSuccess ||
            cudaHostGetDevicePointer((void**)&r.dev, r.host, 0) != cudaSuccess ||
            cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return destroy_and(ABM_ENOMEM);
        }
    char* a = b->arena;
    int k = 0;
    auto at = [&](void) { return (void*)(a + lay.off[k++]); };
    Buffers& B = b->B;
    B.pm[0] = (int4*)at();
    B.pm[1] = (int4*)at();
    B.apar[0] = (uint32_t*)at();
    B.apar[1] = (uint32_t*)at();
    B.rk = (uint32_t*)at();
    B.acc = (uint64_t*)at();
    B.props = (uint2*)at();
    B.pflag = (uint8_t*)at();
    B.xpm = (int4*)at();
    B.xrk = (uint32_t*)at();
    B.bseg = (uint2*)at();
    B.bofs = (uint32_t*)at();
    B.bsrt = (uint32_t*)at();
    B.btofs = (uint32_t*)at();
    B.cnt = (uint32_t*)at();
    B.start = (uint32_t*)at();
    B.tcnt = (uint32_t*)at();
    B.tsum = (uint32_t*)at();
    B.sims = (SimDev*)at();
    B.models = (ModelDev*)at();
    B.counts = (uint64_t*)at();
    B.digests = (uint64_t*)at();
    B.live = (uint64_t*)at();
    B.live_stride = b->max_sims * 512u;
    B.mons = (MonDev*)at();
    B.mon_w = (int32_t*)at();
    B.mon_acc = (uint64_t*)at();
    B.mon_trace = (int64_t*)at();
    int16_t* ztab = (int16_t*)at();
    B.ztab = ztab;
    B.ctl = (Ctl*)at();
    b->staging = (uint32_t*)at();
    B.cap_agents = b->cap_agents;
    B.cap_extras = b->cap_agents / 2 + 1;
    B.cap_cells = b->cap_cells;
    B.bquota = births;
    B.max_sims = b->max_sims;
    B.n_tiles_max = (uint32_t)((b->cap_cells + kTile - 1) / kTile);
    b->sims.resize(b->max_sims);
    b->cell_off_host.assign(b->max_sims, 0);

    // launch shapes: grid-stride kernels sized to the resident capacity
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    b->device = dev;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (b->cap_agents + 255) / 256;
    b->L.threads = 256;
    // the move and scatter passes run best with exactly the CTAs that fit at
    // once (a grid-stride loop, no tail wave); the proposal search with one
    // chunk of sorted agents per CTA, so that the hardware balances chunks of
    // unequal work, and chunks large enough to amortise their compaction
    b->L.blocks_agents =
        (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * (uint64_t)move_blocks_per_sm(256)));
    // the move and scatter passes: block size and CTAs per SM from the options
    // (the autotuner's knobs), else as many CTAs as fit, of 128 threads for
    // capacities from 1M to 2M agents and of 256 otherwise: the move pass's 56
    // registers fit nine 128-thread blocks per SM (36 warps) where 256-thread
    // blocks fit four (32 warps); measured 2.4-3.2% faster steps at 1M and
    // 1.5M agents, within +-1.4% (either way) from 50k to 700k.  Above 2M
    // agents the move pass runs in 48 registers, more warps per SM (measured:
    // 16M agents 502 -> 486 us per step, the 64-sim sweep 0.396 -> 0.388 ms);
    // smaller batches keep the 64-register pass, measured faster there (1M
    // agents: the same step, 22.5-23 instead of 24.6 us in the move pass)
    const bool large = b->cap_agents > (2ull << 20);
    const int tm = o->threads_per_block ? (int)o->threads_per_block
                                        : (!large && b->cap_agents >= (1ull << 20) ? 128 : 256);
    b->L.dense_move = large;
    const uint64_t per_sm = o->blocks_per_sm ? o->blocks_per_sm : (uint64_t)move_blocks_per_sm(tm, large);
    b->L.threads_move = tm;
    b->L.blocks_move = (int)std::max<uint64_t>(
        1, std::min<uint64_t>((b->cap_agents + tm - 1) / tm, (uint64_t)sms * per_sm));
    // the live-counting variant holds more registers: its own resident grid
    // (with the other's, 128-thread blocks would leave a second wave)
    const uint64_t per_sm_live = o->blocks_per_sm ? o->blocks_per_sm : (uint64_t)move_blocks_per_sm(tm, large, true);
    b->L.blocks_move_live = (int)std::max<uint64_t>(
        1, std::min<uint64_t>((b->cap_agents + tm - 1) / tm, (uint64_t)sms * per_sm_live));
    // the scatter needs fewer registers than the move pass: on large batches
    // all of its blocks that fit at once (measured: 16M agents 530 -> 512 us
    // per step); up to 2M agents the move pass's grid (the larger grid cost
    // 1M agents about 1 us)
    const uint64_t per_sm_scatter =
        o->blocks_per_sm ? o->blocks_per_sm
                         : (large ? (uint64_t)std::max(scatter_blocks_per_sm(tm), (int)per_sm) : per_sm);
    b->L.blocks_scatter = (int)std::max<uint64_t>(
        1, std::min<uint64_t>((b->cap_agents + tm - 1) / tm, (uint64_t)sms * per_sm_scatter));
    uint64_t chunk = 1024;
    while (chunk < 4096 && chunk * (uint64_t)sms * 8 < b->cap_agents) chunk *= 2;
    if (o->propose_chunk) chunk = o->propose_chunk;
    B.propose_chunk = (uint32_t)chunk;
    b->L.blocks_propose =
        (int)std::max<uint64_t>(1, std::min<uint64_t>((b->cap_agents + chunk - 1) / chunk, (uint64_t)sms * 32));
    // one scan tile per CTA up to 2048 tiles (the hardware overlaps the tiles'
    // load-scan-store chains; each CTA adds up at most 2048 tile counts before
    // its own), contiguous tile ranges per CTA beyond
    b->L.blocks_scan = (int)std::max<uint64_t>(1, std::min<uint64_t>(B.n_tiles_max, 2048));
    b->L.blocks_accept = sms;
    b->L.prefix_kernel = B.n_tiles_max > kDirectTiles;

    std::vector<int16_t> table(65536);
    std::memcpy(table.data(), o->ncdf_table ? o->ncdf_table : default_table(), 2 * 65536);
#undef CU
#define CU(call)                                                      \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) {                                      \
            cuda_fail(b, e_, #call);                                  \
            return destroy_and(ABM_ECUDA);                            \
        }                                                             \
    } while (0)
    CU(prepare_kernels());
    CU(cudaMemsetAsync(b->arena, 0, lay.total, b->stream));
    CU(cudaMemsetAsync(B.acc, 0xFF, 8 * b->cap_agents, b->stream));  // every proposal slot empty
    CU(cudaMemcpyAsync(ztab, table.data(), 2 * 65536, cudaMemcpyHostToDevice, b->stream));
    Ctl c{};
    c.epoch = 1;
    CU(cudaMemcpyAsync(B.ctl, &c, sizeof c, cudaMemcpyHostToDevice, b->stream));
    CU(cudaStreamSynchronize(b->stream));
#undef CU
    if (capture(b) != ABM_OK) {
        cudaGetLastError();
        return destroy_and(ABM_ECUDA);
    }
    *out = b;
    return ABM_OK;
}

#define CU(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(b, e_, #call); \
    } while (0)

// Agents of a restored simulation, in the engine's layout (hidden partners
// travel inside their carriers' records).
struct RestoreSet {
    std::vector<int4> pm;
    std::vector<uint32_t> id, par;
    uint32_t step = 0, next_id = 0;
};

// Convert and check abm_dump records against a compiled model: ids unique
// and below next_id, species/compartment/reaction in range, positions inside
// the domain and in their compartment, every carrier's hidden partner
// present with the matching reaction.
static abm_status restore_set(const Compiled& c, const abm_record* rec, size_t n, uint32_t step,
                              uint32_t next_id, RestoreSet* out, std::string* err) {
    out->step = step;
    out->next_id = next_id;
    std::vector<const abm_record*> sorted(n);
    for (size_t i = 0; i < n; i++) sorted[i] = rec + i;
    std::sort(sorted.begin(), sorted.end(), [](const abm_record* a, const abm_record* b) { return a->id < b->id; });
    auto bad = [&](const char* m) {
        *err = m;
        return ABM_EINVAL;
    };
    const SimDev& g = c.geo;
    auto find = [&](uint32_t id) -> const abm_record* {
        auto it = std::lower_bound(sorted.begin(), sorted.end(), id,
                                   [](const abm_record* r, uint32_t v) { return r->id < v; });
        return it != sorted.end() && (*it)->id == id ? *it : nullptr;
    };
    for (size_t i = 0; i < n; i++) {
        const abm_record& r = *sorted[i];
        if (i && sorted[i - 1]->id == r.id) return bad("restore: duplicate agent id");
        if (r.id >= next_id) return bad("restore: agent id not below next_id");
        if (r.species >= c.dev.n_sp || r.compartment >= c.dev.n_comp) return bad("restore: species or compartment out of range");
        if (r.x < 0 || r.y < 0 || r.z < 0 || r.x > g.ext || r.y > g.ext || r.z > g.ext) return bad("restore: position outside the domain");
        if (r.flags & 2) continue;  // hidden: restored with its carrier
        int64_t d = 0;
        int comp = 0;
        if (g.root_sphere) {
            const int64_t dx = r.x - g.c0[0], dy = r.y - g.c0[1], dz = r.z - g.c0[2];
            if (dx * dx + dy * dy + dz * dz > g.root_r2) return bad("restore: position outside the cell");
        }
        for (int k = 1; k < g.n_comp; k++) {
            const int64_t dx = r.x - g.cc[k][0], dy = r.y - g.cc[k][1], dz = r.z - g.cc[k][2];
            d = dx * dx + dy * dy + dz * dz;
            if (d <= g.cr2[k]) {
                comp = k;
                break;
            }
        }
        if (comp != r.compartment) return bad("restore: compartment does not match the position");
        uint32_t meta = (uint32_t)r.compartment << M_COMP_SHIFT | r.species;
        uint32_t par = kNone;
        if (r.flags & 1) {
            if (r.reaction >= c.dev.n_rx) return bad("restore: reaction out of range");
            const ReactionDev& R = c.dev.rx[r.reaction];
            const bool ra = r.flags & 4;
            if (r.species != (ra ? R.a : R.b) || R.kind != ABM_BIND || (bool)R.carrier_a != ra)
                return bad("restore: carrier does not match its reaction");
            const abm_record* h = find(r.partner);
            if (!h || !(h->flags & 2) || h->partner != r.id || h->reaction != r.reaction ||
                h->species != (ra ? R.b : R.a))
                return bad("restore: a carrier's hidden partner is missing or inconsistent");
            meta |= M_BOUND | (ra ? M_ROLE_A : 0u) | (uint32_t)r.reaction << M_RXN_SHIFT;
            par = r.partner;
        } else if (c.dev.sp[r.species].partner_mask) {
            meta |= M_PROP;
        }
        out->pm.push_back(make_int4(r.x, r.y, r.z, (int)meta));
        out->id.push_back(r.id);
        out->par.push_back(par);
    }
    for (size_t i = 0; i < n; i++) {  // every hidden record belongs to a carrier
        const abm_record& r = *sorted[i];
        if (!(r.flags & 2)) continue;
        const abm_record* car = find(r.partner);
        if (!car || !(car->flags & 1) || car->partner != r.id) return bad("restore: hidden agent without its carrier");
    }
    return ABM_OK;
}

static abm_status add_sim(abm_batch* b, const abm_model* model, uint64_t seed, uint32_t cell_log2, bool restore,
                          const abm_record* rec, size_t n_rec, uint32_t step, uint32_t next_id, int32_t* sim_id) {
    if (!b || !sim_id) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    *sim_id = -1;
    b->live_valid = false;  // the live counts lack the admitted simulation until a step has run
    std::unique_ptr<Compiled> c_owner(new (std::nothrow) Compiled());
    Compiled* c = c_owner.get();
    if (!c) return ABM_ENOMEM;
    std::string msg;
    abm_status st = compile_model(model, c, &msg);
    if (st != ABM_OK) {
        b->err = msg;  // invalid input does not fail the batch
        return st;
    }
    const uint32_t shift = cell_log2 ? cell_log2 : auto_shift(*c);
    if (shift > 30 || (1ll << shift) < c->Rmax) {
        b->err = "grid cell smaller than a reaction radius";
        return ABM_EINVAL;
    }
    const uint64_t ncell = cells_for(*c, shift);
    RestoreSet rs;
    if (restore) {
        st = restore_set(*c, rec, n_rec, step, next_id, &rs, &msg);
        if (st != ABM_OK) {
            b->err = msg;
            return st;
        }
        c->n0 = rs.pm.size();  // agents to place
    }
    Ctl h;
    st = sync_and_check(b, &h);
    if (st != ABM_OK) {
        return st;
    }
    auto free_slot = [&]() -> int32_t {
        for (uint32_t s = 0; s < b->max_sims; s++)
            if (b->sims[s].state == 0) return (int32_t)s;
        return -1;
    };
    // retired sims keep their slot and agents until the next step drops them;
    // when either is needed now, drop them here
    int32_t slot = free_slot();
    bool draining = false;
    for (uint32_t s = 0; s < b->max_sims; s++) draining |= b->sims[s].state == 2;
    if (draining && (slot < 0 || (uint64_t)h.n_buf[h.cur] + c->n0 > b->cap_agents)) {
        st = compact(b, &h);
        if (st != ABM_OK) {
            return st;
        }
        slot = free_slot();
    }
    if (slot < 0 || cells_in_use(b) + ncell > b->cap_cells || (uint64_t)h.n_buf[h.cur] + c->n0 > b->cap_agents) {
        b->err = slot < 0 ? "no free simulation slot"
                 : cells_in_use(b) + ncell > b->cap_cells ? "grid cells exhausted" : "agent capacity exhausted";
        return ABM_ECAPACITY;
    }
    // model table: reuse an identical upload
    int mslot = -1;
    for (size_t m = 0; m < b->model_host.size(); m++)
        if (b->model_refs[m] > 0 && std::memcmp(&b->model_host[m], &c->dev, sizeof(ModelDev)) == 0) {
            mslot = (int)m;
            break;
        }
    if (mslot < 0) {
        for (size_t m = 0; m < b->model_host.size(); m++)
            if (b->model_refs[m] == 0) {
                mslot = (int)m;
                break;
            }
        if (mslot < 0) {
            mslot = (int)b->model_host.size();
            b->model_host.emplace_back();
            b->model_refs.push_back(0);
        }
        b->model_host[mslot] = c->dev;
        CU(cudaMemcpyAsync(&b->B.models[mslot], &c->dev, sizeof(ModelDev), cudaMemcpyHostToDevice, b->stream));
    }
    b->model_refs[mslot]++;
    SimDev sd = c->geo;
    sd.active = 1;
    sd.model = (uint32_t)mslot;
    sd.key0 = (uint32_t)seed;
    sd.key1 = (uint32_t)(seed >> 32);
    sd.step = restore ? rs.step : 0;
    sd.next_id = restore ? rs.next_id : (uint32_t)c->n0;
    sd.shift = shift;
    sd.g = (uint32_t)((c->geo.ext >> shift) + 1);
    sd.n_counts = c->dev.n_counts;
    sd.counts_off = (uint32_t)slot * 512u;
    sd.max_step = 0xFFFFFFFFu;
    auto& hs = b->sims[slot];
    hs.state = 1;
    hs.status = ABM_OK;
    hs.err.clear();
    hs.model_slot = (uint32_t)mslot;
    hs.n_cells = ncell;
    hs.n_counts = c->dev.n_counts;
    hs.shift = shift;
    b->n_sims_used = std::max<uint32_t>(b->n_sims_used, (uint32_t)slot + 1);
    CU(cudaMemcpyAsync(&b->B.sims[slot], &sd, sizeof sd, cudaMemcpyHostToDevice, b->stream));
    CU(cudaMemcpyAsync(b->staging, c->species_end, 4 * kMaxSpecies, cudaMemcpyHostToDevice, b->stream));
    const uint32_t nsu = b->n_sims_used;
    CU(cudaMemcpyAsync(&b->B.ctl->n_sims, &nsu, 4, cudaMemcpyHostToDevice, b->stream));
    std::vector<int4> packed;  // (uploaded asynchronously: alive until the synchronisation below)
    if (restore) {
        const size_t k = rs.pm.size();
        packed.resize(k);
        for (size_t i = 0; i < k; i++) {
            rs.pm[i].w |= (int)((uint32_t)slot << M_SIM_SHIFT);
            packed[i] = repack(rs.pm[i], rs.id[i]);
        }
        if (k) {
            CU(cudaMemcpyAsync(b->B.pm[h.cur] + h.n_buf[h.cur], packed.data(), 16 * k, cudaMemcpyHostToDevice,
                               b->stream));
            CU(cudaMemcpyAsync(b->B.apar[h.cur] + h.n_buf[h.cur], rs.par.data(), 4 * k, cudaMemcpyHostToDevice,
                               b->stream));
        }
    } else {
        CU(launch_init(b->B, b->L, b->stream, (uint32_t)slot, h.n_buf[h.cur], (uint32_t)c->n0, b->staging,
                       c->dev.n_sp));
    }
    const uint32_t n_in = h.n_buf[h.cur] + (uint32_t)c->n0;
    CU(cudaMemcpyAsync(&b->B.ctl->n_buf[h.cur], &n_in, 4, cudaMemcpyHostToDevice, b->stream));
    st = repack_cells(b);  // synchronises (host temporaries above stay alive until then)
    if (st != ABM_OK) return st;
    st = sync_and_check(b);
    if (st != ABM_OK) return st;
    *sim_id = slot;
    return ABM_OK;
}

abm_status abm_batch_add(abm_batch* b, const abm_model* model, uint64_t seed, uint32_t cell_log2, int32_t* sim_id) {
    return add_sim(b, model, seed, cell_log2, false, nullptr, 0, 0, 0, sim_id);
}

abm_status abm_batch_restore(abm_batch* b, const abm_model* model, uint64_t seed, uint32_t cell_log2,
                             const abm_record* records, size_t n_records, uint32_t step, uint32_t next_id,
                             int32_t* sim_id) {
    if (!b || !sim_id || (n_records && !records)) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    return add_sim(b, model, seed, cell_log2, true, records, n_records, step, next_id, sim_id);
}

abm_status abm_batch_remove(abm_batch* b, int32_t sim) {
    if (!b) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    if (sim < 0 || (uint32_t)sim >= b->max_sims || b->sims[sim].state != 1) return ABM_ESTATE;
    if (b->sims[sim].monitor) {
        abm_status st = abm_batch_monitor_clear(b, sim);
        if (st != ABM_OK) return st;
    }
    const uint32_t zero = 0;
    CU(cudaMemcpyAsync(&b->B.sims[sim].active, &zero, 4, cudaMemcpyHostToDevice, b->stream));
    b->sims[sim].state = 2;
    b->live_valid = false;
    b->model_refs[b->sims[sim].model_slot]--;
    return repack_cells(b);
}

// ------------------------------------------------------------------------
// Threshold monitors (one per simulation slot).
abm_status abm_batch_monitor_set(abm_batch* b, int32_t sim, const abm_monitor* m, const int32_t* weights,
                                 size_t n_weights) {
    if (!b || !m || (n_weights && !weights)) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    if (sim < 0 || (uint32_t)sim >= b->max_sims || b->sims[sim].state != 1) return ABM_ESTATE;
    // the last counts entry (next id) is not a count of records
    if (n_weights > b->sims[sim].n_counts - 1 || m->period == 0 || m->step_end <= m->step_begin) {
        b->err = "monitor: weights longer than the counts vector, period 0 or an empty window";
        return ABM_EINVAL;
    }
    for (size_t k = 0; k < n_weights; k++)
        if (weights[k] > (1 << 20) || weights[k] < -(1 << 20)) {
            b->err = "monitor: weights must lie in [-2^20, 2^20]";
            return ABM_EINVAL;
        }
    abm_status st = sync_and_check(b);
    if (st != ABM_OK) return st;
    b->mon_w_host.assign(512, 0);
    std::copy(weights, weights + n_weights, b->mon_w_host.begin());
    MonDev& M = b->mon_host;
    M = MonDev{};
    M.active = 1;
    M.begin = m->step_begin;
    M.end = m->step_end;
    M.period = m->period;
    M.threshold = m->threshold;
    M.above = m->above ? 1u : 0u;
    M.last_step = 0;
    M.first_pass = kNone;
    M.state = -1;
    if (!b->sims[sim].monitor) b->n_monitors++;
    b->sims[sim].monitor = true;
    const uint64_t zero = 0;
    CU(cudaMemcpyAsync(b->B.mon_w + (size_t)sim * 512, b->mon_w_host.data(), 4 * 512, cudaMemcpyHostToDevice,
                       b->stream));
    CU(cudaMemcpyAsync(b->B.mons + sim, &M, sizeof(MonDev), cudaMemcpyHostToDevice, b->stream));
    CU(cudaMemcpyAsync(b->B.mon_acc + sim, &zero, 8, cudaMemcpyHostToDevice, b->stream));
    CU(cudaMemcpyAsync(&b->B.ctl->n_monitors, &b->n_monitors, 4, cudaMemcpyHostToDevice, b->stream));
    return sync_and_check(b);
}

abm_status abm_batch_monitor_clear(abm_batch* b, int32_t sim) {
    if (!b) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    if (sim < 0 || (uint32_t)sim >= b->max_sims || b->sims[sim].state != 1) return ABM_ESTATE;
    if (!b->sims[sim].monitor) return ABM_OK;
    abm_status st = sync_and_check(b);
    if (st != ABM_OK) return st;
    b->sims[sim].monitor = false;
    b->n_monitors--;
    const uint32_t zero = 0;
    CU(cudaMemcpyAsync(&b->B.mons[sim].active, &zero, 4, cudaMemcpyHostToDevice, b->stream));
    CU(cudaMemcpyAsync(&b->B.ctl->n_monitors, &b->n_monitors, 4, cudaMemcpyHostToDevice, b->stream));
    return sync_and_check(b);
}

abm_status abm_batch_monitor_read(abm_batch* b, int32_t sim, abm_monitor_state* out, int64_t* trace, size_t cap,
                                  size_t* n_out) {
    if (!b || !out || (cap && !trace)) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    if (sim < 0 || (uint32_t)sim >= b->max_sims || b->sims[sim].state != 1) return ABM_ESTATE;
    if (!b->sims[sim].monitor) {
        b->err = "monitor: no threshold monitor on this simulation";
        return ABM_ESTATE;
    }
    CU(launch_monitor(b->B, b->L, b->stream, sim));
    MonDev M;
    std::vector<int64_t> ring(kMonTrace);
    CU(cudaMemcpyAsync(&M, b->B.mons + sim, sizeof(MonDev), cudaMemcpyDeviceToHost, b->stream));
    CU(cudaMemcpyAsync(ring.data(), b->B.mon_trace + (size_t)sim * kMonTrace, 8 * kMonTrace,
                       cudaMemcpyDeviceToHost, b->stream));
    abm_status st = sync_and_check(b);
    if (st == ABM_OK) st = sim_status(b, sim);
    if (st != ABM_OK) return st;
    out->value = M.value;
    out->last_step = M.last_step;
    out->first_pass = M.first_pass;
    out->n_evaluated = M.n_eval;
    out->n_passed = M.n_passed;
    out->state = M.state;
    out->reserved = 0;
    // oldest first: the ring holds the last min(n_eval, kMonTrace) values
    const uint32_t kept = std::min<uint32_t>(M.n_eval, kMonTrace);
    if (n_out) *n_out = kept;
    const size_t want = std::min<size_t>(cap, kept);
    for (size_t k = 0; k < want; k++) trace[k] = ring[(M.n_eval - kept + k) % kMonTrace];
    return ABM_OK;
}

abm_status abm_batch_set_max_step(abm_batch* b, int32_t sim, uint32_t max_step) {
    if (!b) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    if (sim < 0 || (uint32_t)sim >= b->max_sims || b->sims[sim].state != 1) return ABM_ESTATE;
    b->max_step_host = max_step;
    CU(cudaMemcpyAsync(&b->B.sims[sim].max_step, &b->max_step_host, 4, cudaMemcpyHostToDevice, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return ABM_OK;
}

abm_status abm_batch_step(abm_batch* b, uint32_t n) {
    if (!b) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    if (const int inj = g_inject_launch_error.exchange(0))
        return cuda_fail(b, (cudaError_t)inj, "cudaGraphLaunch (injected)");
    if (n > 0)
        for (auto& h : b->sims)
            if (h.state == 2) h.state = 0;  // their agents are dropped by this step
    const uint32_t steps = n;
    cudaGraphExec_t g1 = b->live_on ? b->g1_live : b->g1, g8 = b->live_on ? b->g8_live : b->g8;
    while (n >= 8) {
        CU(cudaGraphLaunch(g8, b->stream));
        n -= 8;
    }
    while (n--) CU(cudaGraphLaunch(g1, b->stream));
    if (steps) {
        b->epoch_host += steps;
        b->live_valid = b->live_on != 0;
    }
    return ABM_OK;
}

abm_status abm_batch_profile_step(abm_batch* b, uint32_t n, float* kernel_ms, uint32_t n_kernels) {
    if (!b || !kernel_ms || n_kernels < (uint32_t)kStepKernels) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    if (n > 0)
        for (auto& h : b->sims)
            if (h.state == 2) h.state = 0;
    const int mode = b->live_on != 0;
    if (!b->prof_ev[0])
        for (auto& e : b->prof_ev) CU(cudaEventCreate(&e));
    if (!b->gprof[mode]) {
        cudaStream_t cs;
        CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t el = launch_step_timed(b->B, b->L, cs, b->prof_ev, mode != 0);
            e = cudaStreamEndCapture(cs, &graph);
            if (e == cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gprof[mode], graph, 0);
        if (e == cudaSuccess) e = cudaGraphUpload(b->gprof[mode], b->stream);  // (first replay not slower)
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return cuda_fail(b, e, "profile graph");
    }
    double acc[kStepKernels] = {};
    cudaError_t e = cudaSuccess;
    for (uint32_t s = 0; s < n && e == cudaSuccess; s++) {
        e = cudaGraphLaunch(b->gprof[mode], b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b->prof_ev[kStepKernels]);
        for (int k = 0; k < kStepKernels && e == cudaSuccess; k++) {
            float ms = 0;
            e = cudaEventElapsedTime(&ms, b->prof_ev[k], b->prof_ev[k + 1]);
            if (k != 1 || b->L.prefix_kernel) acc[k] += ms;  // slot 1: k_tile_prefix, large grids only
        }
    }
    if (e != cudaSuccess) return cuda_fail(b, e, "profile step");
    if (n) {
        b->epoch_host += n;
        b->live_valid = b->live_on != 0;
    }
    for (int k = 0; k < kStepKernels; k++) kernel_ms[k] = (float)acc[k];
    return sync_and_check(b);
}

abm_status abm_batch_sync(abm_batch* b) {
    if (!b) return ABM_EINVAL;
    return sync_and_check(b);
}

abm_status abm_batch_sim_status(abm_batch* b, int32_t sim) {
    if (!b) return ABM_EINVAL;
    abm_status st = sync_and_check(b);
    if (st != ABM_OK) return st;
    if (sim < 0 || (uint32_t)sim >= b->max_sims || b->sims[sim].state != 1) return ABM_ESTATE;
    return sim_status(b, sim);
}

abm_status abm_batch_live_agents(abm_batch* b, uint64_t* out) {
    if (!b || !out) return ABM_EINVAL;
    Ctl h;
    abm_status st = sync_and_check(b, &h);
    if (st == ABM_OK) *out = h.n_buf[h.cur];
    return st;
}

static abm_status observe(abm_batch* b, int32_t sim, int want_digest) {
    if (b->failed) return ABM_ESTATE;
    if (sim < 0 || (uint32_t)sim >= b->max_sims || b->sims[sim].state != 1) return ABM_ESTATE;
    CU(cudaMemsetAsync(b->B.counts + (size_t)sim * 512, 0, 8 * 512, b->stream));
    if (want_digest) CU(cudaMemsetAsync(b->B.digests + sim, 0, 8, b->stream));
    CU(launch_observe(b->B, b->L, b->stream, sim, want_digest));
    return ABM_OK;
}

abm_status abm_batch_counts(abm_batch* b, int32_t sim, uint64_t* out, size_t cap, size_t* n_out) {
    if (!b) return ABM_EINVAL;
    abm_status st = observe(b, sim, 0);
    if (st != ABM_OK) return st;
    const size_t n = b->sims[sim].n_counts;
    if (n_out) *n_out = n;
    // through the pinned staging copy: the copy stays asynchronous, and one
    // synchronisation covers it and the error check
    if (out && cap) CU(cudaMemcpyAsync(b->h_counts, b->B.counts + (size_t)sim * 512, 8 * std::min(cap, n),
                                       cudaMemcpyDeviceToHost, b->stream));
    st = sync_and_check(b);
    if (st == ABM_OK) st = sim_status(b, sim);
    if (st == ABM_OK && out && cap) std::memcpy(out, b->h_counts, 8 * std::min(cap, n));
    if (st == ABM_OK && out && cap < n) return ABM_EINVAL;
    return st;
}

abm_status abm_batch_counts_begin(abm_batch* b, int32_t sim, uint32_t slot) {
    if (!b || slot >= ABM_READ_SLOTS || b->rs[slot].pending) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    if (sim < 0 || (uint32_t)sim >= b->max_sims || b->sims[sim].state != 1) return ABM_ESTATE;
    // live counts of the last step's result when they hold the current state,
    // else a pass over the agents
    const uint64_t* src = b->B.live + (size_t)((b->epoch_host - 1u) & 1u) * b->B.live_stride;
    if (!b->live_valid) {
        abm_status st = observe(b, sim, 0);
        if (st != ABM_OK) return st;
        src = b->B.counts;
    }
    auto& r = b->rs[slot];
    r.n = b->sims[sim].n_counts;
    r.sim = sim;
    // one block writes the counts and the control words into the pinned slot;
    // stream order keeps a later reset of these counts behind it
    CU(launch_readout(src + (size_t)sim * 512, r.n, b->B.ctl, r.dev, b->stream));
    CU(cudaEventRecord(r.done, b->stream));
    r.pending = true;
    return ABM_OK;
}

abm_status abm_batch_live_counts(abm_batch* b, int on) {
    if (!b) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    if (on && !b->g1_live) {  // the step graphs with the counting move pass
        CU(cudaStreamSynchronize(b->stream));
        abm_status st = capture(b, true);
        if (st != ABM_OK) return st;
    }
    b->live_on = on ? 1u : 0u;
    b->live_valid = false;  // from the next step on
    CU(cudaMemsetAsync(b->B.live, 0, 2 * 8 * (size_t)b->B.live_stride, b->stream));
    CU(cudaMemcpyAsync(&b->B.ctl->live_counts, &b->live_on, 4, cudaMemcpyHostToDevice, b->stream));
    return ABM_OK;
}

abm_status abm_batch_counts_finish(abm_batch* b, uint32_t slot, uint64_t* out, size_t cap, size_t* n_out) {
    if (!b || slot >= ABM_READ_SLOTS || !b->rs[slot].pending) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    auto& r = b->rs[slot];
    r.pending = false;
    CU(cudaEventSynchronize(r.done));
    Ctl h;
    std::memcpy(&h, r.host + 512, sizeof(Ctl));
    abm_status st = check_ctl(b, h);
    if (st == ABM_OK && r.sim >= 0 && (uint32_t)r.sim < b->max_sims) st = sim_status(b, r.sim);
    if (st != ABM_OK) return st;
    if (n_out) *n_out = r.n;
    if (out && cap) std::memcpy(out, r.host, 8 * std::min<size_t>(cap, r.n));
    return out && cap < r.n ? ABM_EINVAL : ABM_OK;
}

abm_status abm_batch_digest(abm_batch* b, int32_t sim, uint64_t* out) {
    if (!b || !out) return ABM_EINVAL;
    abm_status st = observe(b, sim, 1);
    if (st != ABM_OK) return st;
    CU(cudaMemcpyAsync(b->h_counts, b->B.digests + sim, 8, cudaMemcpyDeviceToHost, b->stream));
    st = sync_and_check(b);
    if (st == ABM_OK) st = sim_status(b, sim);
    if (st == ABM_OK) *out = b->h_counts[0];
    return st;
}

abm_status abm_batch_dump(abm_batch* b, int32_t sim, abm_record* out, size_t cap, size_t* n_out) {
    if (!b) return ABM_EINVAL;
    if (b->failed) return ABM_ESTATE;
    if (sim < 0 || (uint32_t)sim >= b->max_sims || b->sims[sim].state != 1) return ABM_ESTATE;
    Ctl h;
    abm_status st = sync_and_check(b, &h);
    if (st == ABM_OK) st = sim_status(b, sim);
    if (st != ABM_OK) return st;
    const uint32_t dcap = (uint32_t)std::min<uint64_t>(2ull * h.n_buf[h.cur] + 1, 0xFFFFFFF0ull);
    void* d = nullptr;
    CU(cudaMalloc(&d, (size_t)dcap * 24));
    const uint32_t zero = 0;
    cudaError_t e = cudaMemcpyAsync(&b->B.ctl->dump_n, &zero, 4, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = launch_dump(b->B, b->L, b->stream, sim, d, dcap);
    uint32_t n = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n, &b->B.ctl->dump_n, 4, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    std::vector<uint4> lo;
    std::vector<uint2> hi;
    if (e == cudaSuccess) {
        lo.resize(n);
        hi.resize(n);
        e = cudaMemcpy(lo.data(), d, (size_t)n * 16, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(hi.data(), (char*)d + (size_t)dcap * 16, (size_t)n * 8, cudaMemcpyDeviceToHost);
    }
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(b, e, "dump");
    if (n_out) *n_out = n;
    if (!out) return ABM_OK;
    if (cap < n) return ABM_EINVAL;
    std::vector<abm_record> recs(n);
    for (uint32_t i = 0; i < n; i++) {
        abm_record& r = recs[i];
        r.id = lo[i].x;
        r.species = (uint8_t)(lo[i].y & 0xFF);
        r.compartment = (uint8_t)((lo[i].y >> 8) & 0xFF);
        r.flags = (uint8_t)((lo[i].y >> 16) & 0xFF);
        r.reaction = (uint8_t)(lo[i].y >> 24);
        r.x = (int32_t)lo[i].z;
        r.y = (int32_t)lo[i].w;
        r.z = (int32_t)hi[i].x;
        r.partner = hi[i].y;
    }
    std::sort(recs.begin(), recs.end(), [](const abm_record& p, const abm_record& q) { return p.id < q.id; });
    std::memcpy(out, recs.data(), (size_t)n * sizeof(abm_record));
    return ABM_OK;
}

const char* abm_batch_last_error(const abm_batch* b) { return b ? b->err.c_str() : "null handle"; }

void abm_batch_destroy(abm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->g1) cudaGraphExecDestroy(b->g1);
    if (b->g8) cudaGraphExecDestroy(b->g8);
    if (b->g1_live) cudaGraphExecDestroy(b->g1_live);
    if (b->g8_live) cudaGraphExecDestroy(b->g8_live);
    for (auto& g : b->gprof)
        if (g) cudaGraphExecDestroy(g);
    for (auto& e : b->prof_ev)
        if (e) cudaEventDestroy(e);
    if (b->own_arena && b->arena) cudaFree(b->arena);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->h_counts) cudaFreeHost(b->h_counts);
    for (auto& r : b->rs) {
        if (r.host) cudaFreeHost(r.host);
        if (r.done) cudaEventDestroy(r.done);
    }
    delete b;
}

// ---------------- single simulation = a batch of one ----------------
size_t abm_arena_bytes(const abm_model* model, const abm_options* opt) {
    std::unique_ptr<Compiled> c_owner(new (std::nothrow) Compiled());
    Compiled* c = c_owner.get();
    if (!c) return 0;
    std::string msg;
    size_t bytes = 0;
    if (compile_model(model, c, &msg) == ABM_OK) {
        const uint32_t shift = opt && opt->cell_log2 ? opt->cell_log2 : auto_shift(*c);
        const uint64_t cap = opt && opt->capacity_agents ? opt->capacity_agents : c->n0 + c->n0 / 4 + 65536;
        abm_batch_options o{};
        o.capacity_agents = cap;
        o.capacity_cells = cells_for(*c, shift);
        o.max_sims = 1;
        o.births_per_step = opt ? opt->births_per_step : 0;
        bytes = abm_batch_arena_bytes(&o);
    }
    return bytes;
}

abm_status abm_model_grid(const abm_model* model, uint32_t cell_log2, uint32_t* shift_out, uint64_t* cells_out) {
    if (!shift_out || !cells_out) return ABM_EINVAL;
    std::unique_ptr<Compiled> c_owner(new (std::nothrow) Compiled());
    Compiled* c = c_owner.get();
    if (!c) return ABM_ENOMEM;
    std::string msg;
    abm_status st = compile_model(model, c, &msg);
    if (st == ABM_OK) {
        const uint32_t shift = cell_log2 ? cell_log2 : auto_shift(*c);
        if (shift > 30 || (1ll << shift) < c->Rmax) {
            st = ABM_EINVAL;
        } else {
            *shift_out = shift;
            *cells_out = cells_for(*c, shift);
        }
    }
    return st;
}

abm_status abm_create(const abm_model* model, uint64_t seed, const abm_options* opt, abm_sim** out) {
    if (!out) return ABM_EINVAL;
    *out = nullptr;
    std::unique_ptr<Compiled> c_owner(new (std::nothrow) Compiled());
    Compiled* c = c_owner.get();
    if (!c) return ABM_ENOMEM;
    std::string msg;
    abm_status st = compile_model(model, c, &msg);
    const uint32_t shift = st == ABM_OK ? (opt && opt->cell_log2 ? opt->cell_log2 : auto_shift(*c)) : 0;
    const uint64_t n0 = c->n0;
    const uint64_t cells = st == ABM_OK ? cells_for(*c, shift) : 0;
    const bool small_cell = st == ABM_OK && (1ll << shift) < c->Rmax;
    if (st != ABM_OK || small_cell || shift > 30) return ABM_EINVAL;
    abm_batch_options o{};
    o.capacity_agents = opt && opt->capacity_agents ? opt->capacity_agents : n0 + n0 / 4 + 65536;
    if (o.capacity_agents < n0) return ABM_ECAPACITY;
    o.capacity_cells = cells;
    o.max_sims = 1;
    o.births_per_step = opt ? opt->births_per_step : 0;
    o.arena = opt ? opt->arena : nullptr;
    o.arena_bytes = opt ? opt->arena_bytes : 0;
    o.stream = opt ? opt->stream : nullptr;
    o.ncdf_table = opt ? opt->ncdf_table : nullptr;
    abm_batch* b = nullptr;
    st = abm_batch_create(&o, &b);
    if (st != ABM_OK) return st;
    b->single = true;
    int32_t id = -1;
    st = abm_batch_add(b, model, seed, shift, &id);
    if (st != ABM_OK) {
        abm_batch_destroy(b);
        return st;
    }
    abm_sim* s = new (std::nothrow) abm_sim();
    if (!s) {
        abm_batch_destroy(b);
        return ABM_ENOMEM;
    }
    s->b = b;
    s->id = id;
    *out = s;
    return ABM_OK;
}

abm_status abm_restore(const abm_model* model, uint64_t seed, const abm_options* opt, const abm_record* records,
                       size_t n_records, uint32_t step, uint32_t next_id, abm_sim** out) {
    if (!out || (n_records && !records)) return ABM_EINVAL;
    *out = nullptr;
    std::unique_ptr<Compiled> c_owner(new (std::nothrow) Compiled());
    Compiled* c = c_owner.get();
    if (!c) return ABM_ENOMEM;
    std::string msg;
    abm_status st = compile_model(model, c, &msg);
    const uint32_t shift = st == ABM_OK ? (opt && opt->cell_log2 ? opt->cell_log2 : auto_shift(*c)) : 0;
    const uint64_t cells = st == ABM_OK ? cells_for(*c, shift) : 0;
    const bool small_cell = st == ABM_OK && (1ll << shift) < c->Rmax;
    if (st != ABM_OK || small_cell || shift > 30) return ABM_EINVAL;
    abm_batch_options o{};
    o.capacity_agents = opt && opt->capacity_agents ? opt->capacity_agents : n_records + n_records / 4 + 65536;
    o.capacity_cells = cells;
    o.max_sims = 1;
    o.births_per_step = opt ? opt->births_per_step : 0;
    o.arena = opt ? opt->arena : nullptr;
    o.arena_bytes = opt ? opt->arena_bytes : 0;
    o.stream = opt ? opt->stream : nullptr;
    o.ncdf_table = opt ? opt->ncdf_table : nullptr;
    abm_batch* b = nullptr;
    st = abm_batch_create(&o, &b);
    if (st != ABM_OK) return st;
    b->single = true;
    int32_t id = -1;
    st = abm_batch_restore(b, model, seed, shift, records, n_records, step, next_id, &id);
    if (st != ABM_OK) {
        abm_batch_destroy(b);
        return st;
    }
    abm_sim* sim = new (std::nothrow) abm_sim();
    if (!sim) {
        abm_batch_destroy(b);
        return ABM_ENOMEM;
    }
    sim->b = b;
    sim->id = id;
    *out = sim;
    return ABM_OK;
}

abm_status abm_step(abm_sim* s, uint32_t n) { return s ? abm_batch_step(s->b, n) : ABM_EINVAL; }
abm_status abm_counts(abm_sim* s, uint64_t* out, size_t cap, size_t* n_out) {
    return s ? abm_batch_counts(s->b, s->id, out, cap, n_out) : ABM_EINVAL;
}
abm_status abm_counts_begin(abm_sim* s, uint32_t slot) {
    return s ? abm_batch_counts_begin(s->b, s->id, slot) : ABM_EINVAL;
}
abm_status abm_counts_finish(abm_sim* s, uint32_t slot, uint64_t* out, size_t cap, size_t* n_out) {
    return s ? abm_batch_counts_finish(s->b, slot, out, cap, n_out) : ABM_EINVAL;
}
abm_status abm_live_counts(abm_sim* s, int on) { return s ? abm_batch_live_counts(s->b, on) : ABM_EINVAL; }
abm_status abm_digest(abm_sim* s, uint64_t* out) { return s ? abm_batch_digest(s->b, s->id, out) : ABM_EINVAL; }
abm_status abm_dump(abm_sim* s, abm_record* out, size_t cap, size_t* n_out) {
    return s ? abm_batch_dump(s->b, s->id, out, cap, n_out) : ABM_EINVAL;
}
abm_status abm_sync(abm_sim* s) { return s ? abm_batch_sync(s->b) : ABM_EINVAL; }
abm_status abm_monitor_set(abm_sim* s, const abm_monitor* m, const int32_t* weights, size_t n_weights) {
    return s ? abm_batch_monitor_set(s->b, s->id, m, weights, n_weights) : ABM_EINVAL;
}
abm_status abm_monitor_clear(abm_sim* s) { return s ? abm_batch_monitor_clear(s->b, s->id) : ABM_EINVAL; }
abm_status abm_monitor_read(abm_sim* s, abm_monitor_state* out, int64_t* trace, size_t cap, size_t* n_out) {
    return s ? abm_batch_monitor_read(s->b, s->id, out, trace, cap, n_out) : ABM_EINVAL;
}
abm_status abm_profile_step(abm_sim* s, uint32_t n, float* kernel_ms, uint32_t n_kernels) {
    return s ? abm_batch_profile_step(s->b, n, kernel_ms, n_kernels) : ABM_EINVAL;
}
const char* abm_kernel_name(uint32_t k) {
    static const char* names[] = {"k_move", "k_tile_prefix", "k_scan", "k_scatter", "k_propose", "k_accept"};
    return k < (uint32_t)kStepKernels ? names[k] : nullptr;
}
abm_status abm_step_index(abm_sim* s, uint32_t* out) {
    if (!s || !out) return ABM_EINVAL;
    abm_batch* b = s->b;
    abm_status st = sync_and_check(b);
    if (st != ABM_OK) return st;
    CU(cudaMemcpy(out, &b->B.sims[s->id].step, 4, cudaMemcpyDeviceToHost));
    return ABM_OK;
}
abm_status abm_grid_cells(abm_sim* s, uint64_t* out) {
    if (!s || !out) return ABM_EINVAL;
    *out = s->b->sims[s->id].n_cells;
    return ABM_OK;
}
const char* abm_last_error(const abm_sim* s) { return s ? abm_batch_last_error(s->b) : "null handle"; }
void abm_destroy(abm_sim* s) {
    if (!s) return;
    abm_batch_destroy(s->b);
    delete s;
}

void abm_debug_inject_launch_error(int cuda_error) { g_inject_launch_error.store(cuda_error); }

abm_status abm_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n) {
    if (!ctr || !key || !out) return ABM_EINVAL;
    std::string msg;
    if (check_device(&msg) != ABM_OK) return ABM_EDEVICE;
    uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc((void**)&dc, 16 * n + 16);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dk, 8 * n + 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dout, 16 * n + 16);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, 16 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, 8 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_debug_philox(dc, dk, dout, n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 16 * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return e == cudaSuccess ? ABM_OK : ABM_ECUDA;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Internal view of a simulation handle for the library's other translation
// units (no effect on any state).
namespace abm {
bool internal_view(abm_sim* s, Buffers* B, Launch* L, cudaStream_t* stream, int32_t* sim, std::string** err,
                   int* device) {
    if (!s || !s->b || s->b->failed) return false;
    *B = s->b->B;
    *L = s->b->L;
    *stream = s->b->stream;
    *sim = s->id;
    *err = &s->b->err;
    *device = s->b->device;
    return true;
}

// A CUDA failure seen by another translation unit: the handle becomes
// destroy-only, exactly as after a failure inside this file.
abm_status internal_cuda_fail(abm_sim* s, cudaError_t e, const char* where) {
    return cuda_fail(s->b, e, where);
}
}  // namespace abm
