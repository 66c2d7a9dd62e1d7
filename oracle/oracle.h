/*
 * oracle.h — serial CPU reference simulator for the molecule-agent step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load, call or link this.  The
 * product library never includes this header and shares no code with it.
 *
 * The method (paper, Sec. 2 "Materials and Methods"): every molecule is an
 * agent (a sphere) that diffuses by Brownian motion, binds or reacts with a
 * partner found by spatial proximity, releases products after a turnover time,
 * is born from an expressor at a fixed rate, degrades, and migrates between
 * compartments at a translocation rate (Sec. 2, footnote 1 and the four
 * molecule classes; Sec. 3.4 for compartments and expression).  The paper
 * defers all mechanics to earlier work; the integer readings used here are
 * listed at the top of oracle.c.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_CONVERT = 0, ORC_BIND = 1 };
enum { ORC_CUBE = 0, ORC_SPHERE = 1 };

typedef struct {
    uint32_t initial_count;
    double   D_um2_s;        /* diffusion coefficient, um^2/s               */
    int32_t  compartment;    /* where the initial agents are placed         */
    double   p_cross;        /* per attempted membrane crossing             */
    double   p_uni;          /* first-order conversion / death per step     */
    int32_t  uni_to;         /* -1 = death                                  */
    double   p_emit;         /* expressor birth probability per step        */
    int32_t  emit_species;   /* -1 = none                                   */
} orc_species;

typedef struct {
    int32_t a, b;            /* a proposes to b                             */
    int32_t kind;            /* ORC_CONVERT | ORC_BIND                      */
    int32_t prod_a, prod_b;  /* species after the event; -1 = dies          */
    double  radius_nm;       /* contact radius                              */
    double  p_bind;          /* pair Bernoulli applied to eligible contacts */
    double  p_release;       /* per step, bound complexes only              */
} orc_reaction;

typedef struct {
    int32_t shape;           /* ORC_CUBE | ORC_SPHERE                       */
    double  size_um;         /* cube edge or sphere diameter                */
    int32_t parent;          /* -1 for the root, 0 for a child sphere       */
    double  center_um[3];    /* child: centre offset from the root centre   */
} orc_compartment;

/* One 24-byte dump record per agent (hidden agents included), id-sorted. */
typedef struct {
    uint32_t id;
    uint8_t  sp, comp, flags, rxn;   /* flags: 1 bound carrier, 2 hidden, 4 role a */
    int32_t  x, y, z;
    uint32_t partner;
} orc_record;

typedef struct orc_sim orc_sim;

/* Returns NULL and writes a message into err on invalid input. */
orc_sim* orc_create(const orc_species* sp, uint32_t n_sp,
                    const orc_reaction* rx, uint32_t n_rx,
                    const orc_compartment* comp, uint32_t n_comp,
                    double dt_s, double unit_nm, uint64_t seed,
                    int brute_force, char* err, size_t err_len);
void     orc_step(orc_sim* s, uint32_t n);
size_t   orc_counts(const orc_sim* s, uint64_t* out, size_t cap);
uint64_t orc_digest(const orc_sim* s);
size_t   orc_dump(const orc_sim* s, orc_record* out, size_t cap);
size_t   orc_n_agents(const orc_sim* s);
uint32_t orc_step_index(const orc_sim* s);
/* Replace the Gaussian table before the first step (the table is data, and
   the caller may supply its own).  Returns 0, or -1 when the largest entry
   would step past the domain, in which case the table is left unchanged. */
int      orc_set_table(orc_sim* s, const int16_t* table65536);
void     orc_destroy(orc_sim* s);

/* Building blocks exposed for the pins. */
void     orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void     orc_ncdf_table(int16_t* out65536);
int64_t  orc_gauss_step(int16_t z, uint64_t m);
uint64_t orc_threshold(double p);
uint64_t orc_mult(double D_um2_s, double dt_s, double unit_nm);

#ifdef __cplusplus
}
#endif
#endif
