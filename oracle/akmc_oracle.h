/*
 * akmc_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, serial, float64 reference implementation of rejection-free
 * vacancy AKMC on a periodic bcc Fe-Cu-Ni-Mn lattice (the classical AKMC
 * that AtomWorld, arXiv 2604.24091, accelerates: every migration direction
 * of every vacancy is enumerated and rated, one event is selected in
 * proportion to its rate and the clock advances by an amount inversely
 * proportional to the total rate; Sec. "Current State of the Art",
 * Sec. "Compute-Centric Reformulation", Eq. 8).
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load this library.  It shares no source with the CUDA library; the two
 * meet only through the seeded inputs (synth/).
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * (published Philox known answers, brute-force full-lattice energies,
 * detailed balance, closed forms for pure Fe, exact conservation, Boltzmann
 * occupancy on a tiny lattice, library connected components).
 */
#ifndef AKMC_ORACLE_H
#define AKMC_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ETRAPPED = 5, ORC_ENUMERIC = 6 };

typedef struct {
    double eps1[25], eps2[25];      /* pair energies [a*5+b], species Fe,Cu,Ni,Mn,V */
    double E0[4];                   /* barrier at dE=0 of the jumping species      */
    double nu;                      /* attempt frequency, 1/s                      */
    double a;                       /* lattice constant, Angstrom                  */
    double r_cut;                   /* EAM cutoff, Angstrom                        */
    int32_t n_r;                    /* points of phi/f tables (0: no EAM)          */
    int32_t n_rho;                  /* points of F tables                          */
    double rho_h;                   /* knot spacing of F, a power of two           */
    const double* phi_tab;          /* [10][n_r][2] value, d/dr                    */
    const double* f_tab;            /* [4][n_r][2]                                 */
    const double* F_tab;            /* [4][n_rho][2] value, d/drho                 */
} orc_model;

typedef struct {
    int32_t L, n_vac;
    double frac[3];                 /* Cu, Ni, Mn fractions of all 2L^3 sites      */
    double T;
    int32_t model;                  /* 0 pair, 1 EAM                               */
    uint64_t seed, uid;
} orc_desc;

typedef struct orc_voxel orc_voxel;

/* Create a voxel and place species with the Philox placement stream. */
orc_voxel* orc_create(const orc_desc* d, const orc_model* m, int* status);
void orc_destroy(orc_voxel* v);
/* Replace the lattice (vacancy slot k sits at vac_pos[k]); clock and counter set too. */
int orc_load(orc_voxel* v, const uint8_t* species, const int32_t* vac_pos, int32_t n_vac,
             double t_hi, double t_lo, uint64_t n_events);
/* Run n events (stops early if trapped or on a numeric error); log gets
 * 8*slot+dir and dt_log the residence time of the state before each event
 * (both nullable, capacity n). */
int orc_step(orc_voxel* v, uint64_t n, int32_t* log, double* dt_log);
/* Synchronous sublattice schedule: n_supersteps supersteps k0, k0+1, ...; sectors
 * of S^3 cells (S even, >= 8, dividing L), window T seconds per octant (the
 * clock advances T/8 per superstep); reverse != 0 takes
 * the sectors of a superstep in descending order (the result must not change).
 * events[st] (nullable) gets the events made in superstep st. */
int orc_step_sublattice(orc_voxel* v, uint64_t k0, uint32_t n_supersteps, int32_t S, double T, int32_t reverse,
                        uint64_t* events);
int orc_get(const orc_voxel* v, uint8_t* species, int32_t* vac_pos, int32_t* vac_disp,
            double* rates, double* dE, double* t_hi, double* t_lo, uint64_t* n_events);
int32_t orc_n_sites(const orc_voxel* v);
int32_t orc_n_vac(const orc_voxel* v);
double orc_total_rate(const orc_voxel* v);

/* Energies: full-lattice total, local hop dE (a2/a3) and brute-force hop dE. */
double orc_energy(const orc_voxel* v);
double orc_hop_de_local(const orc_voxel* v, int slot, int dir);
double orc_hop_de_brute(const orc_voxel* v, int slot, int dir);
/* Barrier and rate of one hop as the step uses them (rate 0 into a vacancy). */
double orc_hop_rate(const orc_voxel* v, int slot, int dir);
/* Site density rho_i (fixed point, units 2^-24) recomputed from scratch. */
int64_t orc_rho_fixed(const orc_voxel* v, int site);
/* rho_fixed of every site (N entries), from the current lattice. */
void orc_rho_all(const orc_voxel* v, int64_t* out);

/* Debug checks: 1 incremental rates == scratch rates every event,
 * 2 tree selection == linear cumulative scan, 4 stored rho == scratch rho,
 * 8 per-atom tracer displacements. */
void orc_set_debug(orc_voxel* v, int flags);
/* [0] rate mismatches, [1] scan disagreements, [2] disagreements beyond the
 * tie margin 1e-12, [3] rho mismatches, [4] events checked */
void orc_debug_counts(const orc_voxel* v, uint64_t out[5]);
/* Sum over atoms of |unwrapped displacement|^2 in half-unit^2 (flag 8). */
double orc_tracer_r2(const orc_voxel* v);

/* Cu clusters: connected components of Cu under 1nn+2nn (mode 0) or 1nn (mode 1).
 * hist[8] bins sizes {1,2,3,4,5-9,10-19,20-49,>=50}; sizes_out (nullable,
 * capacity N) receives every cluster size; returns the number of clusters. */
int32_t orc_cluster_hist(const orc_voxel* v, int mode, int64_t hist[8], int32_t* sizes_out);

/* Shell constants of the EAM model: phi[10][5] (eV), f[4][5] fixed point 2^-24. */
int orc_shell_constants(const orc_model* m, double phi[50], int64_t fq[20]);
/* F_a(rho) from the Hermite table at a fixed-point density; *err set if clamped. */
double orc_embed(const orc_model* m, int a, int64_t rho_fixed, int* err);

/* Philox4x32-10 block and the two uniforms of event n. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_event_uniforms(uint64_t seed, uint64_t uid, uint64_t n, double* u1, double* u2);

#ifdef __cplusplus
}
#endif
#endif
