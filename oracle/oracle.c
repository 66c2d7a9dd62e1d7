/*
 * oracle.c — plain, serial, slow reference for the molecule-agent time step.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Agents live in one array sorted by
 * id; every phase is a plain loop over that array in ascending id.  Nothing
 * here is blocked, fused or reordered beyond what the step definition states.
 *
 * What the paper fixes (Sec. 2, "Materials and Methods"; Sec. 3.4):
 *   - each molecule is an agent with a position that diffuses (Brownian motion
 *     with a per-species diffusion coefficient);
 *   - agents react when spatially close: active species bind substrates or
 *     inhibitors, a bound complex releases its products after a time set by
 *     the turnover number (here a per-step release probability);
 *   - expressors produce new molecules at a fixed rate; molecules degrade;
 *   - molecules move between compartments at a translocation rate.
 *
 * Where the paper is silent, the following integer readings define the step
 * (both this oracle and the CUDA engine implement them, independently):
 *
 *   RNG      Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  key = seed
 *            (low word, high word).  Counters: agent event block
 *            (id, t, 1, 0); agent move block (id, t, 0, 0); pair block
 *            (min id, max id, t, 1); initial placement (id, attempt, 0, 2).
 *   Events   thr(p) = floor(p * 2^32) (a 64-bit value); an event fires iff the
 *            32-bit draw u < thr(p).  p = 1 always fires, p = 0 never.
 *   Gauss    Z[i] = round(4096 * inv_Phi((i + 1/2) / 65536)), i in [0, 65536),
 *            exactly antisymmetric.  Index = top 16 bits of a Philox word.
 *            M = llround(sqrt(2 D dt) * 1000 / unit_nm * 2^20); the step is
 *            d = sgn(Z) * ((|Z| * M + 2^31) >> 32)  (units of unit_nm).
 *   Phases   P1 events, P2 move, P3 neighbour lists, P4 proposals,
 *            P5 accept + apply, P6 births; each phase reads the state left by
 *            the previous one.
 *   P1       carrier: release iff e0 < thr_rel[rxn]; the pair separates, each
 *            takes its product species (-1 dies), the hidden partner appears
 *            at the carrier's position and compartment.  Free agent: convert
 *            (or die) iff e1 < thr_uni; otherwise emit a child iff
 *            e2 < thr_emit.  Bound agents are immune to conversion/emission.
 *            Only agents free or carrying at the start of P1 take P1 events.
 *   P2       free agents and carriers with M > 0 move.  Cube root: mirror
 *            (x < 0 -> -1 - x; x > L -> 2L + 1 - x).  Sphere root: a move that ends
 *            outside (|p-c|^2 > r^2) is rejected.  A move that changes the
 *            compartment (child spheres, inclusive boundary) is a crossing
 *            attempt: kept iff m3 < thr_cross[species], else rejected.
 *   P4       a free agent of a reaction's species a proposes to the free agent
 *            b (same compartment, reaction (a,b) defined, dist^2 <= R^2,
 *            pair draw < thr_bind) minimising (dist^2, id_b).
 *   P5       acc[b] = min over proposers of (dist^2 << 32 | id_a).  Edge a->b
 *            is final iff acc[b] names a and nobody proposed to a.  CONVERT:
 *            a -> prod_a, b -> prod_b (-1 dies).  BIND: the reactant with the
 *            smaller D carries the complex (tie: a); the other is hidden and
 *            sits at the carrier's position.
 *   P6       children of P1 emitters get ids next_id + k, k ranking parents by
 *            id; they appear at the parent's end-of-P2 position/compartment.
 *   Units    every physical-to-integer conversion is evaluated left to right
 *            in IEEE double and rounded half away from zero (llround).
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define NONE32 0xFFFFFFFFu
#define EMPTY64 0xFFFFFFFFFFFFFFFFull
#define MAX_SP 64
#define MAX_RX 255
#define MAX_COMP 4

typedef struct {
    uint32_t id;
    int      sp, comp;
    int      bound, hidden, role_a, dead;
    int      rxn;
    uint32_t partner;
    int32_t  x, y, z;
} agent_t;

typedef struct {
    int      parent_index;  /* index into the agent array at P1 time */
    int      sp;
    int32_t  x, y, z;
    int      comp;
} birth_t;

struct orc_sim {
    int n_sp, n_rx, n_comp;
    orc_species     sp[MAX_SP];
    orc_reaction    rx[MAX_RX];
    orc_compartment cm[MAX_COMP];
    uint64_t thr_uni[MAX_SP], thr_emit[MAX_SP], thr_cross[MAX_SP], M[MAX_SP];
    uint64_t thr_bind[MAX_RX], thr_rel[MAX_RX];
    int64_t  R[MAX_RX];
    int      rx_of[MAX_SP][MAX_SP];
    int      proposes[MAX_SP];
    int64_t  Rmax;
    int      root_sphere;
    int64_t  ext;            /* positions lie in [0, ext] on every axis */
    int64_t  root_r, c0[3];  /* root sphere radius and the root centre  */
    int64_t  child_r[MAX_COMP], child_c[MAX_COMP][3];
    int16_t  Z[65536];
    uint32_t key[2];
    int      brute;
    agent_t* a;
    size_t   n, cap;
    uint32_t next_id, t;
};

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from the round function and key schedule in Salmon et al.
 * SC'11: two 32x32->64 multiplies per round, Weyl key bumps between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(const orc_sim* s, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t out[4]) {
    uint32_t ctr[4] = {w0, w1, w2, w3};
    orc_philox4x32_10(ctr, s->key, out);
}

/* ------------------------------------------------------------------ */
/* The standard normal CDF from the complementary error function. */
static double normal_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Inverse CDF by plain bisection on the lower half (p < 1/2), where erfc is
 * accurate to a few ulp relative; the upper half is the mirror image. */
void orc_ncdf_table(int16_t* out) {
    for (int i = 0; i < 32768; i++) {
        double p = (i + 0.5) / 65536.0;
        double lo = -40.0, hi = 0.0;
        for (int it = 0; it < 400; it++) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (normal_cdf(mid) < p) lo = mid; else hi = mid;
        }
        double q = 0.5 * (lo + hi);                /* q < 0 */
        int16_t mag = (int16_t)floor(-4096.0 * q + 0.5);
        out[i] = (int16_t)-mag;
        out[65535 - i] = mag;
    }
}

int64_t orc_gauss_step(int16_t z, uint64_t m) {
    if (z >= 0) return (int64_t)(((uint64_t)z * m + 0x80000000ull) >> 32);
    return -(int64_t)(((uint64_t)(-(int32_t)z) * m + 0x80000000ull) >> 32);
}

uint64_t orc_threshold(double p) { return (uint64_t)floor(p * 4294967296.0); }

uint64_t orc_mult(double D_um2_s, double dt_s, double unit_nm) {
    double sigma_delta = sqrt(2.0 * D_um2_s * dt_s) * 1000.0 / unit_nm;
    return (uint64_t)llround(sigma_delta * 1048576.0);
}

static int64_t to_delta(double um, double unit_nm) { return llround(um * 1000.0 / unit_nm); }

/* ------------------------------------------------------------------ */
static int64_t dist2(int64_t x, int64_t y, int64_t z, const int64_t c[3]) {
    int64_t dx = x - c[0], dy = y - c[1], dz = z - c[2];
    return dx * dx + dy * dy + dz * dz;
}

/* Compartment containing the point; -1 if outside a spherical root. */
static int locate(const orc_sim* s, int64_t x, int64_t y, int64_t z) {
    if (s->root_sphere && dist2(x, y, z, s->c0) > s->root_r * s->root_r) return -1;
    for (int k = 1; k < s->n_comp; k++)
        if (dist2(x, y, z, s->child_c[k]) <= s->child_r[k] * s->child_r[k]) return k;
    return 0;
}

static int valid_p(double p) { return p >= 0.0 && p <= 1.0; }

static int fail(char* err, size_t len, const char* msg) {
    if (err && len) snprintf(err, len, "%s", msg);
    return 0;
}

static int compile_model(orc_sim* s, const orc_species* sp, uint32_t n_sp, const orc_reaction* rx,
                         uint32_t n_rx, const orc_compartment* cm, uint32_t n_comp, double dt,
                         double unit, char* err, size_t el) {
    if (n_sp < 1 || n_sp > MAX_SP) return fail(err, el, "species count out of range");
    if (n_rx > MAX_RX) return fail(err, el, "too many reactions");
    if (n_comp < 1 || n_comp > MAX_COMP) return fail(err, el, "compartment count out of range");
    if (!(dt > 0) || !(unit > 0)) return fail(err, el, "dt and unit must be positive");
    s->n_sp = (int)n_sp; s->n_rx = (int)n_rx; s->n_comp = (int)n_comp;
    memcpy(s->sp, sp, n_sp * sizeof *sp);
    if (n_rx) memcpy(s->rx, rx, n_rx * sizeof *rx);
    memcpy(s->cm, cm, n_comp * sizeof *cm);

    /* geometry: compartment 0 is the root; the others are child spheres */
    if (cm[0].parent != -1) return fail(err, el, "compartment 0 must be the root");
    if (cm[0].shape == ORC_CUBE) {
        s->root_sphere = 0;
        s->ext = to_delta(cm[0].size_um, unit);
        s->c0[0] = s->c0[1] = s->c0[2] = s->ext / 2;
    } else if (cm[0].shape == ORC_SPHERE) {
        s->root_sphere = 1;
        s->root_r = llround(cm[0].size_um * 1000.0 / unit / 2.0);
        s->ext = 2 * s->root_r;
        s->c0[0] = s->c0[1] = s->c0[2] = s->root_r;
    } else {
        return fail(err, el, "unknown root shape");
    }
    if (s->ext < 2 || s->ext > (1 << 30)) return fail(err, el, "root size out of range");
    for (int k = 1; k < (int)n_comp; k++) {
        if (cm[k].parent != 0 || cm[k].shape != ORC_SPHERE) return fail(err, el, "child must be a sphere in the root");
        s->child_r[k] = llround(cm[k].size_um * 1000.0 / unit / 2.0);
        for (int d = 0; d < 3; d++) s->child_c[k][d] = s->c0[d] + to_delta(cm[k].center_um[d], unit);
        int64_t r = s->child_r[k];
        if (r < 1) return fail(err, el, "child sphere too small");
        if (s->root_sphere) {
            int64_t room = s->root_r - r;
            if (room < 0 || dist2(s->child_c[k][0], s->child_c[k][1], s->child_c[k][2], s->c0) > room * room)
                return fail(err, el, "child sphere leaves the root");
        } else {
            for (int d = 0; d < 3; d++)
                if (s->child_c[k][d] - r < 0 || s->child_c[k][d] + r > s->ext) return fail(err, el, "child sphere leaves the root");
        }
        for (int j = 1; j < k; j++) {
            int64_t rr = s->child_r[j] + r;
            if (dist2(s->child_c[k][0], s->child_c[k][1], s->child_c[k][2], s->child_c[j]) <= rr * rr)
                return fail(err, el, "child spheres overlap");
        }
    }

    orc_ncdf_table(s->Z);
    int zmax = 0;
    for (int i = 0; i < 65536; i++) zmax = abs(s->Z[i]) > zmax ? abs(s->Z[i]) : zmax;

    for (int i = 0; i < (int)n_sp; i++) {
        const orc_species* q = &sp[i];
        if (!(q->D_um2_s >= 0) || !valid_p(q->p_cross) || !valid_p(q->p_uni) || !valid_p(q->p_emit))
            return fail(err, el, "species parameter out of range");
        if (q->compartment < 0 || q->compartment >= (int)n_comp) return fail(err, el, "bad species compartment");
        if (q->uni_to < -1 || q->uni_to >= (int)n_sp || q->emit_species < -1 || q->emit_species >= (int)n_sp)
            return fail(err, el, "unknown species referenced");
        s->M[i] = orc_mult(q->D_um2_s, dt, unit);
        if (s->M[i] >= (1ull << 32)) return fail(err, el, "diffusion step too large");
        if (orc_gauss_step((int16_t)zmax, s->M[i]) > s->ext) return fail(err, el, "diffusion step exceeds the domain");
        s->thr_uni[i] = orc_threshold(q->p_uni);
        s->thr_emit[i] = q->emit_species >= 0 ? orc_threshold(q->p_emit) : 0;
        s->thr_cross[i] = orc_threshold(q->p_cross);
    }
    for (int i = 0; i < MAX_SP; i++) {
        s->proposes[i] = 0;
        for (int j = 0; j < MAX_SP; j++) s->rx_of[i][j] = -1;
    }
    s->Rmax = 0;
    for (int r = 0; r < (int)n_rx; r++) {
        const orc_reaction* q = &rx[r];
        if (q->a < 0 || q->a >= (int)n_sp || q->b < 0 || q->b >= (int)n_sp) return fail(err, el, "unknown reactant");
        if (q->a == q->b) return fail(err, el, "A+A reactions are not supported");
        if (q->kind != ORC_CONVERT && q->kind != ORC_BIND) return fail(err, el, "unknown reaction kind");
        if (q->prod_a < -1 || q->prod_a >= (int)n_sp || q->prod_b < -1 || q->prod_b >= (int)n_sp)
            return fail(err, el, "unknown product");
        if (!valid_p(q->p_bind) || !valid_p(q->p_release)) return fail(err, el, "reaction probability out of range");
        if (s->rx_of[q->a][q->b] >= 0 || s->rx_of[q->b][q->a] >= 0) return fail(err, el, "duplicate reactant pair");
        s->R[r] = llround(q->radius_nm / unit);
        if (s->R[r] < 1 || s->R[r] > 30000) return fail(err, el, "reaction radius out of range");
        s->thr_bind[r] = orc_threshold(q->p_bind);
        s->thr_rel[r] = orc_threshold(q->p_release);
        s->rx_of[q->a][q->b] = r;
        s->proposes[q->a] = 1;
        if (s->R[r] > s->Rmax) s->Rmax = s->R[r];
    }
    return 1;
}

static int grow(orc_sim* s, size_t need) {
    if (need <= s->cap) return 1;
    size_t cap = s->cap ? s->cap : 1024;
    while (cap < need) cap *= 2;
    agent_t* p = realloc(s->a, cap * sizeof *p);
    if (!p) return 0;
    s->a = p; s->cap = cap;
    return 1;
}

orc_sim* orc_create(const orc_species* sp, uint32_t n_sp, const orc_reaction* rx, uint32_t n_rx,
                    const orc_compartment* cm, uint32_t n_comp, double dt_s, double unit_nm,
                    uint64_t seed, int brute_force, char* err, size_t err_len) {
    orc_sim* s = calloc(1, sizeof *s);
    if (!s) return NULL;
    if (!compile_model(s, sp, n_sp, rx, n_rx, cm, n_comp, dt_s, unit_nm, err, err_len)) {
        free(s);
        return NULL;
    }
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
    s->brute = brute_force;
    uint64_t total = 0;
    for (int i = 0; i < s->n_sp; i++) total += sp[i].initial_count;
    if (total >= NONE32 || !grow(s, (size_t)total + 1)) {
        fail(err, err_len, "too many agents");
        free(s->a); free(s);
        return NULL;
    }
    /* Initial placement: ids species-major; each agent draws uniform integer
     * coordinates in [0, ext] until they fall in its species' compartment. */
    uint32_t id = 0;
    for (int i = 0; i < s->n_sp; i++) {
        for (uint32_t k = 0; k < sp[i].initial_count; k++, id++) {
            int placed = 0;
            for (uint32_t attempt = 0; attempt < (1u << 24) && !placed; attempt++) {
                uint32_t w[4];
                draw(s, id, attempt, 0, 2, w);
                int64_t x = (int64_t)(((uint64_t)w[0] * (uint64_t)(s->ext + 1)) >> 32);
                int64_t y = (int64_t)(((uint64_t)w[1] * (uint64_t)(s->ext + 1)) >> 32);
                int64_t z = (int64_t)(((uint64_t)w[2] * (uint64_t)(s->ext + 1)) >> 32);
                if (locate(s, x, y, z) != sp[i].compartment) continue;
                agent_t* A = &s->a[s->n++];
                memset(A, 0, sizeof *A);
                A->id = id; A->sp = i; A->comp = sp[i].compartment;
                A->rxn = -1; A->partner = NONE32;
                A->x = (int32_t)x; A->y = (int32_t)y; A->z = (int32_t)z;
                placed = 1;
            }
            if (!placed) {
                fail(err, err_len, "could not place an agent in its compartment");
                free(s->a); free(s);
                return NULL;
            }
        }
    }
    s->next_id = id;
    s->t = 0;
    return s;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->a);
    free(s);
}

/* Array index of the agent with this id (the array is sorted by id). */
static size_t find(const orc_sim* s, uint32_t id) {
    size_t lo = 0, hi = s->n;
    while (lo < hi) {
        size_t mid = (lo + hi) / 2;
        if (s->a[mid].id < id) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int is_free(const agent_t* A) { return !A->dead && !A->bound && !A->hidden; }

static void set_species_or_die(agent_t* A, int sp) {
    if (sp < 0) A->dead = 1; else A->sp = sp;
}

/* ---------------- P1: first-order events ---------------- */
static void phase_events(orc_sim* s, birth_t** births, size_t* nb) {
    size_t n = s->n;
    char* active = malloc(n ? n : 1);
    for (size_t i = 0; i < n; i++) active[i] = !s->a[i].dead && !s->a[i].hidden;
    *births = malloc((n ? n : 1) * sizeof **births);
    *nb = 0;
    for (size_t i = 0; i < n; i++) {
        if (!active[i]) continue;
        agent_t* A = &s->a[i];
        /* the draw is only read by carriers and by species with an event */
        if (!A->bound && s->thr_uni[A->sp] == 0 && s->thr_emit[A->sp] == 0) continue;
        uint32_t e[4];
        draw(s, A->id, s->t, 1, 0, e);
        if (A->bound) {
            if ((uint64_t)e[0] < s->thr_rel[A->rxn]) {
                const orc_reaction* r = &s->rx[A->rxn];
                agent_t* H = &s->a[find(s, A->partner)];
                int carrier_prod = A->role_a ? r->prod_a : r->prod_b;
                int hidden_prod = A->role_a ? r->prod_b : r->prod_a;
                H->x = A->x; H->y = A->y; H->z = A->z; H->comp = A->comp;
                A->bound = 0; H->hidden = 0;
                A->role_a = H->role_a = 0;
                A->rxn = H->rxn = -1;
                A->partner = H->partner = NONE32;
                set_species_or_die(A, carrier_prod);
                set_species_or_die(H, hidden_prod);
            }
        } else if ((uint64_t)e[1] < s->thr_uni[A->sp]) {
            set_species_or_die(A, s->sp[A->sp].uni_to);
        } else if ((uint64_t)e[2] < s->thr_emit[A->sp]) {
            birth_t* b = &(*births)[(*nb)++];
            b->parent_index = (int)i;
            b->sp = s->sp[A->sp].emit_species;
        }
    }
    free(active);
}

/* ---------------- P2: Brownian move with boundaries ---------------- */
/* Fold about the half-integer walls -1/2 and L+1/2, which maps the integer
 * line onto [0, L] while preserving the counting measure (the uniform
 * distribution on [0, L] is exactly stationary under symmetric steps). */
static int64_t mirror(int64_t v, int64_t L) {
    if (v < 0) return -v - 1;
    if (v > L) return 2 * L + 1 - v;
    return v;
}

static void phase_move(orc_sim* s) {
    for (size_t i = 0; i < s->n; i++) {
        agent_t* A = &s->a[i];
        if (A->dead || A->hidden) continue;
        uint64_t M = s->M[A->sp];
        if (M == 0) continue;
        uint32_t m[4];
        draw(s, A->id, s->t, 0, 0, m);
        int64_t x = A->x + orc_gauss_step(s->Z[m[0] >> 16], M);
        int64_t y = A->y + orc_gauss_step(s->Z[m[1] >> 16], M);
        int64_t z = A->z + orc_gauss_step(s->Z[m[2] >> 16], M);
        if (!s->root_sphere) {
            x = mirror(x, s->ext); y = mirror(y, s->ext); z = mirror(z, s->ext);
        }
        int c = locate(s, x, y, z);
        if (c < 0) continue;                                   /* left the cell: rejected */
        if (c != A->comp) {
            if ((uint64_t)m[3] >= s->thr_cross[A->sp]) continue; /* membrane: rejected */
            A->comp = c;
        }
        A->x = (int32_t)x; A->y = (int32_t)y; A->z = (int32_t)z;
    }
    /* a hidden agent travels inside its carrier */
    for (size_t i = 0; i < s->n; i++) {
        agent_t* A = &s->a[i];
        if (!A->bound) continue;
        agent_t* H = &s->a[find(s, A->partner)];
        H->x = A->x; H->y = A->y; H->z = A->z; H->comp = A->comp;
    }
}

/* ---------------- P3/P4: neighbour lists and proposals ---------------- */
typedef struct {
    int64_t h, g;     /* cell edge and cells per axis */
    int32_t* head;
    int32_t* next;
} cells_t;

static void build_cells(const orc_sim* s, cells_t* c) {
    int64_t h = (s->ext + 100) / 100;        /* about 100 cells per axis */
    if (h < s->Rmax) h = s->Rmax;
    if (h < 1) h = 1;
    c->h = h;
    c->g = s->ext / h + 1;
    size_t ncell = (size_t)(c->g * c->g * c->g);
    c->head = malloc(ncell * sizeof(int32_t));
    c->next = malloc((s->n ? s->n : 1) * sizeof(int32_t));
    for (size_t k = 0; k < ncell; k++) c->head[k] = -1;
    for (size_t i = 0; i < s->n; i++) {
        const agent_t* A = &s->a[i];
        c->next[i] = -1;
        if (!is_free(A)) continue;
        size_t k = (size_t)(((A->z / h) * c->g + A->y / h) * c->g + A->x / h);
        c->next[i] = c->head[k];
        c->head[k] = (int32_t)i;
    }
}

static void consider(const orc_sim* s, size_t i, size_t j, uint64_t* best, int64_t* best_j) {
    const agent_t* A = &s->a[i];
    const agent_t* B = &s->a[j];
    if (j == i || !is_free(B) || B->comp != A->comp) return;
    int r = s->rx_of[A->sp][B->sp];
    if (r < 0) return;
    int64_t dx = (int64_t)A->x - B->x, dy = (int64_t)A->y - B->y, dz = (int64_t)A->z - B->z;
    int64_t d2 = dx * dx + dy * dy + dz * dz;
    if (d2 > s->R[r] * s->R[r]) return;
    uint32_t lo = A->id < B->id ? A->id : B->id, hi = A->id < B->id ? B->id : A->id;
    uint32_t u[4];
    draw(s, lo, hi, s->t, 1, u);
    if ((uint64_t)u[0] >= s->thr_bind[r]) return;
    uint64_t key = ((uint64_t)d2 << 32) | B->id;
    if (key < *best) { *best = key; *best_j = (int64_t)j; }
}

static void phase_propose(orc_sim* s, int64_t* target, uint64_t* prop_key) {
    cells_t c = {0};
    if (!s->brute) build_cells(s, &c);
    for (size_t i = 0; i < s->n; i++) {
        const agent_t* A = &s->a[i];
        target[i] = -1;
        if (!is_free(A) || !s->proposes[A->sp]) continue;
        uint64_t best = EMPTY64;
        int64_t best_j = -1;
        if (s->brute) {
            for (size_t j = 0; j < s->n; j++) consider(s, i, j, &best, &best_j);
        } else {
            int64_t cx = A->x / c.h, cy = A->y / c.h, cz = A->z / c.h;
            for (int64_t z = cz - 1; z <= cz + 1; z++)
                for (int64_t y = cy - 1; y <= cy + 1; y++)
                    for (int64_t x = cx - 1; x <= cx + 1; x++) {
                        if (x < 0 || y < 0 || z < 0 || x >= c.g || y >= c.g || z >= c.g) continue;
                        for (int32_t j = c.head[(z * c.g + y) * c.g + x]; j >= 0; j = c.next[j])
                            consider(s, i, (size_t)j, &best, &best_j);
                    }
        }
        if (best_j >= 0) {
            target[i] = best_j;
            prop_key[i] = (best & 0xFFFFFFFF00000000ull) | A->id;
        }
    }
    free(c.head);
    free(c.next);
}

/* ---------------- P5: acceptance and reaction application ---------------- */
static void apply(orc_sim* s, size_t ia, size_t ib) {
    agent_t* A = &s->a[ia];
    agent_t* B = &s->a[ib];
    int r = s->rx_of[A->sp][B->sp];
    const orc_reaction* q = &s->rx[r];
    if (q->kind == ORC_CONVERT) {
        set_species_or_die(A, q->prod_a);
        set_species_or_die(B, q->prod_b);
        return;
    }
    int carrier_is_a = !(s->sp[B->sp].D_um2_s < s->sp[A->sp].D_um2_s);
    agent_t* C = carrier_is_a ? A : B;
    agent_t* H = carrier_is_a ? B : A;
    C->bound = 1; C->rxn = r; C->partner = H->id; C->role_a = carrier_is_a;
    H->hidden = 1; H->rxn = r; H->partner = C->id; H->role_a = !carrier_is_a;
    H->x = C->x; H->y = C->y; H->z = C->z; H->comp = C->comp;
}

static void phase_accept(orc_sim* s, const int64_t* target, const uint64_t* prop_key) {
    size_t n = s->n;
    uint64_t* acc = malloc((n ? n : 1) * sizeof *acc);
    for (size_t i = 0; i < n; i++) acc[i] = EMPTY64;
    for (size_t i = 0; i < n; i++)
        if (target[i] >= 0 && prop_key[i] < acc[target[i]]) acc[target[i]] = prop_key[i];
    /* decide every edge before applying any of them */
    char* final_edge = calloc(n ? n : 1, 1);
    for (size_t i = 0; i < n; i++) {
        if (target[i] < 0) continue;
        size_t b = (size_t)target[i];
        if ((uint32_t)acc[b] == s->a[i].id && acc[i] == EMPTY64) final_edge[i] = 1;
    }
    for (size_t i = 0; i < n; i++)
        if (final_edge[i]) apply(s, i, (size_t)target[i]);
    free(final_edge);
    free(acc);
}

/* ---------------- one full step ---------------- */
static void one_step(orc_sim* s) {
    birth_t* births;
    size_t nb;
    phase_events(s, &births, &nb);
    phase_move(s);
    for (size_t k = 0; k < nb; k++) {          /* parent's end-of-P2 place */
        const agent_t* P = &s->a[births[k].parent_index];
        births[k].x = P->x; births[k].y = P->y; births[k].z = P->z; births[k].comp = P->comp;
    }
    size_t n = s->n;
    int64_t* target = malloc((n ? n : 1) * sizeof *target);
    uint64_t* prop_key = malloc((n ? n : 1) * sizeof *prop_key);
    phase_propose(s, target, prop_key);
    phase_accept(s, target, prop_key);
    free(target);
    free(prop_key);

    /* P6: births in ascending parent id (P1 ran in id order) */
    grow(s, s->n + nb);
    for (size_t k = 0; k < nb; k++) {
        agent_t* A = &s->a[s->n++];
        memset(A, 0, sizeof *A);
        A->id = s->next_id++;
        A->sp = births[k].sp; A->comp = births[k].comp;
        A->rxn = -1; A->partner = NONE32;
        A->x = births[k].x; A->y = births[k].y; A->z = births[k].z;
    }
    free(births);
    /* drop the dead, keeping id order */
    size_t w = 0;
    for (size_t i = 0; i < s->n; i++)
        if (!s->a[i].dead) s->a[w++] = s->a[i];
    s->n = w;
    s->t++;
}

void orc_step(orc_sim* s, uint32_t n) {
    for (uint32_t k = 0; k < n; k++) one_step(s);
}

/* ---------------- observation ---------------- */
size_t orc_counts(const orc_sim* s, uint64_t* out, size_t cap) {
    size_t need = (size_t)s->n_sp * s->n_comp + s->n_rx + 1;
    if (cap < need) return need;
    memset(out, 0, need * sizeof *out);
    for (size_t i = 0; i < s->n; i++) {
        const agent_t* A = &s->a[i];
        if (is_free(A)) out[A->sp * s->n_comp + A->comp]++;
        else if (A->bound) out[(size_t)s->n_sp * s->n_comp + A->rxn]++;
    }
    out[need - 1] = s->next_id;
    return need;
}

static void record_of(const agent_t* A, orc_record* R) {
    R->id = A->id;
    R->sp = (uint8_t)A->sp;
    R->comp = (uint8_t)A->comp;
    R->flags = (uint8_t)((A->bound ? 1 : 0) | (A->hidden ? 2 : 0) | (A->role_a ? 4 : 0));
    R->rxn = A->rxn < 0 ? 0xFF : (uint8_t)A->rxn;
    R->x = A->x; R->y = A->y; R->z = A->z;
    R->partner = A->partner;
}

/* MurmurHash3 64-bit finaliser (Appleby). */
static uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

/* Order-independent digest: the wrapping sum of a hash of every record, plus
 * a hash of (step, next_id). */
uint64_t orc_digest(const orc_sim* s) {
    uint64_t sum = 0;
    for (size_t i = 0; i < s->n; i++) {
        orc_record R;
        record_of(&s->a[i], &R);
        uint64_t h = fmix64((uint64_t)R.id | (uint64_t)R.sp << 32 | (uint64_t)R.comp << 40 |
                            (uint64_t)R.flags << 48 | (uint64_t)R.rxn << 56);
        h = fmix64(h ^ ((uint64_t)(uint32_t)R.x | (uint64_t)(uint32_t)R.y << 32));
        h = fmix64(h ^ ((uint64_t)(uint32_t)R.z | (uint64_t)R.partner << 32));
        sum += h;
    }
    return sum + fmix64((uint64_t)s->t | (uint64_t)s->next_id << 32);
}

size_t orc_dump(const orc_sim* s, orc_record* out, size_t cap) {
    if (cap < s->n) return s->n;
    for (size_t i = 0; i < s->n; i++) record_of(&s->a[i], &out[i]);
    return s->n;
}

size_t orc_n_agents(const orc_sim* s) { return s->n; }
uint32_t orc_step_index(const orc_sim* s) { return s->t; }

int orc_set_table(orc_sim* s, const int16_t* table) {
    int zmax = 0;
    for (int i = 0; i < 65536; i++) zmax = abs(table[i]) > zmax ? abs(table[i]) : zmax;
    for (int i = 0; i < s->n_sp; i++)
        if ((int64_t)(((uint64_t)zmax * s->M[i] + 0x80000000ull) >> 32) > s->ext) return -1;
    memcpy(s->Z, table, sizeof(s->Z));
    return 0;
}
