/*
 * akmc.h -- C ABI of the GB300 (sm_103a) vacancy AKMC library (libakmc.so).
 *
 * Rejection-free atomistic kinetic Monte Carlo of vacancy-mediated diffusion
 * on periodic bcc Fe-Cu-Ni-Mn voxels: the classical AKMC that AtomWorld
 * (arXiv 2604.24091) accelerates.  Per event and voxel it enumerates and
 * rates every 1nn migration of every vacancy (Sec. "Compute-Centric
 * Reformulation": all migration directions of each vacancy), keeps the rate
 * sums in a per-voxel binary tree, selects one event in proportion to its
 * rate from a counter-based Philox stream, applies the swap and advances a
 * compensated float64 clock by -ln(u)/Gamma_tot (time step inversely
 * proportional to the total rate, Sec. "Current State of the Art").  Rates
 * are Arrhenius (Eq. 8) with a KRA barrier; hops into a vacancy are masked
 * out (the admissibility mask of Eq. 1) and all events of a voxel compete
 * in one global selection (Eq. 2).  Voxels are independent periodic boxes
 * (Sec. "Mesoscopic Voxel-Parallel Formulation"), which is the batch axis.
 *
 * Conventions
 *  - Lattice: site s = ((z*L + y)*L + x)*2 + b, x,y,z in [0,L) cells, b = 0
 *    corner / 1 body centre; half-unit coordinates (2x+b, 2y+b, 2z+b) mod 2L.
 *    Species codes (uint8): Fe 0, Cu 1, Ni 2, Mn 3, vacancy 4.
 *  - Hop direction of a vacancy: dir = (dx<0) + 2(dy<0) + 4(dz<0) for the
 *    1nn vector (+-1,+-1,+-1) in half units; event index = 8*slot + dir.
 *  - Device memory is owned by the caller: every device buffer the library
 *    uses lives in one caller-allocated workspace (for example a torch uint8
 *    tensor).  The library never calls cudaMalloc/cudaFree; it allocates only
 *    small host-side bookkeeping (including pinned staging for targets).
 *  - Streams are passed as opaque pointers (a cudaStream_t; NULL = legacy
 *    default stream).  Calls are stream-ordered and return without waiting,
 *    except akmc_read_state, akmc_sync_status and akmc_cluster_hist, which
 *    synchronise the given stream.
 *  - Errors: every call returns an akmc_status; the text of the last error
 *    of the calling thread is available from akmc_last_error().  Per-voxel
 *    device status words report trapped voxels and numeric errors.  The
 *    library never aborts the process.
 */
#ifndef AKMC_H
#define AKMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct akmc_batch akmc_batch;   /* opaque, owned by the library */
typedef void* akmc_stream;              /* a cudaStream_t */

typedef enum {
    AKMC_OK = 0,
    AKMC_EINVAL = 1,    /* invalid argument or descriptor                         */
    AKMC_ENOMEM = 2,    /* workspace smaller than akmc_workspace_bytes()          */
    AKMC_ECUDA = 3,     /* a CUDA runtime call failed (message in last_error)     */
    AKMC_ETIMEOUT = 4,  /* a bounded device wait gave up (sublattice readiness)  */
    AKMC_ETRAPPED = 5,  /* voxel total rate is 0: no admissible event             */
    AKMC_ENUMERIC = 6   /* density outside the embedding table, or NaN/Inf rate   */
} akmc_status;

enum { AKMC_PAIR = 0, AKMC_EAM = 1 };          /* energy model            */
enum { AKMC_FP64 = 0, AKMC_SPLIT = 1 };        /* EAM arithmetic          */

/* One voxel.  Species counts are n_s = floor(frac_s * 2L^3 + 0.5) for
 * s = Cu, Ni, Mn; n_vac vacancies; Fe is the balance.  Placement draws sites
 * from the Philox placement stream (key = seed, counter word3 has its top
 * bit set) by sequential rejection: vacancies first (slot = placement order),
 * then Cu, Ni, Mn.  Requirements: pair model L >= 3, EAM L >= 4, L <= 1024,
 * 2L^3 < 2^31, 1 <= n_vac <= 256, T > 0. */
typedef struct {
    int32_t L;
    int32_t n_vac;
    double frac[3];
    double T;              /* K */
    int32_t model;         /* AKMC_PAIR or AKMC_EAM */
    int32_t precision;     /* EAM only: AKMC_FP64 or AKMC_SPLIT (FP32 embedding, exact fixed-point + FP64 assembly) */
    uint64_t seed;         /* Philox key */
    uint64_t uid;          /* voxel id: Philox counter words 2-3 (event stream independent of batching) */
} akmc_voxel_desc;

/* Energy model shared by all voxels of a batch (host pointers; copied at create).
 * Pair model: E = 1/2 sum_i sum_{j in N1(i)} eps1[s_i][s_j] + 1/2 sum_i sum_{j in N2(i)} eps2[s_i][s_j],
 *   species order Fe,Cu,Ni,Mn,V; every eps must be a multiple of 2^-24 eV with
 *   |eps| < 4 eV (exact sums).  Hop dE is the exact change of E.
 * EAM: E = sum_{i != V} [F_{s_i}(rho_i) + 1/2 sum_{j in S(i), j != V} phi_{s_i s_j}(r_ij)],
 *   rho_i = sum_{j in S(i), j != V} f_{s_j}(r_ij), S = the 58 sites within r_cut.
 *   phi/f are tabulated on r_k = k*r_cut/(n_r-1), F on rho_k = k*rho_h
 *   (rho_h a power of two in [2^-24, 1]), each as (value, derivative) pairs
 *   evaluated by cubic Hermite interpolation.  f at the 5 shell radii is
 *   rounded to a multiple of 2^-24 (densities are exact fixed-point sums).
 * Barrier Ea = max(0, dE, E0[A] + dE/2) for the jumping species A;
 * rate = nu * exp(-Ea/(kB*T)), kB = 8.617333262e-5 eV/K. */
typedef struct {
    double eps1[25], eps2[25];
    double E0[4];
    double nu;
    double a;              /* lattice constant, Angstrom */
    double r_cut;          /* EAM cutoff, Angstrom (must lie between the 5th and 6th shells) */
    int32_t n_r, n_rho;    /* table lengths (0 when no voxel uses EAM) */
    double rho_h;
    const double* phi_tab; /* [10][n_r][2], pair index of a<=b: a*(7-a)/2 + b */
    const double* f_tab;   /* [4][n_r][2] */
    const double* F_tab;   /* [4][n_rho][2] */
} akmc_model;

/* Host-side view of one voxel; any pointer may be NULL (not copied). */
typedef struct {
    uint8_t* species;      /* [2L^3]                                          */
    int32_t* vac_pos;      /* [n_vac] site of each vacancy slot               */
    int32_t* vac_disp;     /* [3 n_vac] unwrapped displacement, half units    */
    double* rates;         /* [8 n_vac] hop rates (1/s), event order          */
    double* dE;            /* [8 n_vac] hop energy changes (eV), 0 into a vacancy */
    int32_t* event_log;    /* [event_log_capacity] ring: entry n % cap = 8*slot+dir of event n */
    double t_hi, t_lo;     /* simulated time = t_hi + t_lo (s)                */
    uint64_t n_events;     /* events executed so far (Philox event counter)   */
    int32_t status;        /* akmc_status of the voxel                        */
    int32_t L, n_vac;
} akmc_state;

/* Bytes of device workspace a batch needs (0 and last_error set if the
 * descriptors or model are invalid).  Pure host computation. */
size_t akmc_workspace_bytes(const akmc_voxel_desc* descs, int32_t n_voxels,
                            const akmc_model* model, int32_t event_log_capacity);

/* Lay the batch out in dev_workspace (>= akmc_workspace_bytes), upload the
 * model and descriptors, place species on the device (a1) and build densities,
 * rates and rate trees (akmc_compute_rates).  Stream-ordered. */
akmc_status akmc_create_batch(const akmc_voxel_desc* descs, int32_t n_voxels,
                              const akmc_model* model, int32_t event_log_capacity,
                              void* dev_workspace, size_t workspace_bytes,
                              akmc_stream stream, akmc_batch** out);

/* Full rebuild of every voxel: EAM densities from the lattice (fixed-point,
 * exact), then the 8 rates of every vacancy and the rate trees. */
akmc_status akmc_compute_rates(akmc_batch* batch, akmc_stream stream);

/* Run n_events[v] further events on every voxel v (n_voxels entries).  A host
 * array is copied before return and sets the processing order (largest
 * expected work first); a device array is copied on the stream (device to
 * device) and the processing order of the previous call is kept (voxel order
 * before any host call).  One persistent launch steps all voxels;
 * a voxel stops early when trapped or on a numeric error.  Results do not
 * depend on the batch composition or launch shape: each voxel's stream is
 * Philox(seed, (n, uid)). */
akmc_status akmc_step_n(akmc_batch* batch, const uint64_t* n_events, akmc_stream stream);

/* The two halves of akmc_step_n, for CUDA-graph capture and chunked serving:
 * akmc_set_targets copies n_events (host or device, n_voxels entries, as for
 * akmc_step_n) and the processing order into the workspace (stream-ordered;
 * a host array may be reused on return); akmc_launch_step resets the work queue and launches the persistent
 * step kernel with the targets already on the device -- one memset and one
 * kernel, so a stream capture of it replays "run the stored targets again".
 * akmc_launch_step fails with AKMC_EINVAL while rates are out of date after
 * a state load (call akmc_compute_rates first). */
akmc_status akmc_set_targets(akmc_batch* batch, const uint64_t* n_events, akmc_stream stream);
akmc_status akmc_launch_step(akmc_batch* batch, akmc_stream stream);

/* Synchronous sublattice supersteps of one voxel (intra-voxel parallel AKMC,
 * the synchronous form of the sublattice scheme of Sec. 3.2.2).  The voxel is
 * cut into sectors of sector_cells^3 cells (sector_cells even, >= 8, dividing
 * L) and each sector into 8 octants of (sector_cells/2)^3 cells.  Superstep
 * k = superstep0, ..., superstep0 + n_supersteps - 1 evolves octant k mod 8
 * (bit 0: upper half in x, bit 1: y, bit 2: z) of every sector at once: each
 * runs residence-time KMC over the vacancies inside it at the superstep start,
 * with a clock from 0, up to (not including) the first event past window_s
 * seconds; a vacancy that leaves its octant takes no further part in the
 * superstep.  Event i of sector c = (cz (L/Sc) + cy) (L/Sc) + cx in superstep
 * k draws Philox(seed, (i, k, c, 0xC0000000 | uid & 0x3fffffff)).  The voxel
 * clock advances by window_s / 8 per superstep (a cycle of 8 supersteps
 * evolves every region for window_s; Neumaier-compensated), the event
 * counter by the events made; there is no event log.  Sectors of a superstep
 * are independent (events reach 4 half units, active octants are
 * sector_cells + 1 apart), so the result does not depend on their order.  The
 * voxel's rates and tree are rebuilt after the last superstep.  Stream-ordered,
 * no synchronisation; per-voxel status as for akmc_step_n.  AKMC_EINVAL for a
 * bad voxel index, sector size or window (not finite or <= 0). */
akmc_status akmc_step_sublattice(akmc_batch* batch, int32_t voxel, uint64_t superstep0, uint32_t n_supersteps,
                                 int32_t sector_cells, double window_s, akmc_stream stream);

/* The same supersteps with local readiness instead of a global barrier (the
 * asynchronous sublattice scheme of Sec. 3.2.2): one cooperative launch runs
 * all n_supersteps; each sector starts superstep k as soon as its 26
 * neighbouring sectors have finished superstep k - 1 (per-sector counters in
 * the workspace), so distant sectors run different supersteps at the same
 * time.  Neighbouring sectors never run different supersteps concurrently,
 * hence the result is identical to akmc_step_sublattice's (same lattice,
 * positions, counts, clock).  Each readiness wait is bounded (a few
 * seconds); on expiry the voxel's status becomes AKMC_ETIMEOUT.  Arguments,
 * errors and stream semantics as for akmc_step_sublattice; the superstep
 * index is taken modulo 2^32 in both. */
akmc_status akmc_step_sublattice_async(akmc_batch* batch, int32_t voxel, uint64_t superstep0,
                                       uint32_t n_supersteps, int32_t sector_cells, double window_s,
                                       akmc_stream stream);

/* Failure-detection test hook for the asynchronous form: runs supersteps
 * 0 .. n_supersteps-1 like akmc_step_sublattice_async, except that sector
 * stall_sector is never processed and never reports readiness, so the bounded
 * waits of its neighbours run out: the voxel's status becomes AKMC_ETIMEOUT
 * (read with akmc_sync_status) after a few seconds and the device stays usable.
 * The voxel's state is then unspecified.  AKMC_EINVAL for a sector index out
 * of range, otherwise as akmc_step_sublattice_async. */
akmc_status akmc_test_sublattice_stall(akmc_batch* batch, int32_t voxel, uint32_t n_supersteps,
                                       int32_t sector_cells, double window_s, int32_t stall_sector,
                                       akmc_stream stream);

/* Re-seed n voxel slots in place with new descriptors (continuous batching:
 * a finished request's slot takes the next request).  Each new descriptor
 * must keep the slot's L, n_vac and model; T, composition, precision, seed
 * and uid may change (a split-precision voxel in a batch created without one
 * runs the general path: same results, no lattice window).  The slot restarts at event 0 and time 0 with a fresh
 * Philox placement, densities, rate tables, rates and tree; other voxels are
 * untouched.  Stream-ordered with respect to earlier and later launches on
 * the same stream; synchronises the stream before returning. */
akmc_status akmc_reset_voxels(akmc_batch* batch, const int32_t* slots, const akmc_voxel_desc* descs,
                              int32_t n, akmc_stream stream);

/* Copy one voxel's state to host memory; synchronises the stream. */
akmc_status akmc_read_state(akmc_batch* batch, int32_t voxel, akmc_state* out, akmc_stream stream);

/* Copy the EAM site densities of one voxel to host memory: rho[s] for every
 * site s (2L^3 int32, site order as above), in fixed point with unit 2^-24
 * (rho_s = sum over the 58 sites j within the cutoff, j not a vacancy, of
 * f_{sigma_j}(r_sj), each term rounded to that unit: the density that enters
 * the EAM embedding energy).  host_rho is caller-owned.  Fails with
 * AKMC_EINVAL for a pair-model voxel, a NULL pointer, or while the batch's
 * densities are out of date after a state load (call akmc_compute_rates
 * first).  Synchronises the stream. */
akmc_status akmc_read_density(akmc_batch* batch, int32_t voxel, int32_t* host_rho, akmc_stream stream);

/* Replace one voxel's lattice (same L and n_vac), clock and event counter;
 * displacements restart at 0.  The next akmc_step_n or akmc_compute_rates
 * rebuilds rates first.  Host inputs are copied before return. */
akmc_status akmc_load_state(akmc_batch* batch, int32_t voxel, const uint8_t* species,
                            const int32_t* vac_pos, double t_hi, double t_lo,
                            uint64_t n_events, akmc_stream stream);

/* Whole-batch state transfer, for checkpointing and host-fed pipelines.
 * Arrays are concatenated in voxel order: species (sum of 2L^3 bytes),
 * vac_pos and (read only) vac_disp (sum of n_vac, 3 n_vac int32); the
 * per-voxel arrays have n_voxels entries.  Pass pinned host memory for
 * copies that overlap; both calls are stream-ordered and do not synchronise
 * (the host buffers must stay valid until the stream reaches the copies).
 * load_batch_state does no host-side validation of the lattices: each
 * voxel's vac_pos must name its vacancy sites (the next rebuild flags
 * violations).  NULL t_hi/t_lo/n_events leave the clock and counters as they
 * are.  The next akmc_step_n or akmc_compute_rates rebuilds rates first. */
akmc_status akmc_load_batch_state(akmc_batch* batch, const uint8_t* species, const int32_t* vac_pos,
                                  const double* t_hi, const double* t_lo, const uint64_t* n_events,
                                  akmc_stream stream);
akmc_status akmc_read_batch_state(akmc_batch* batch, uint8_t* species, int32_t* vac_pos, int32_t* vac_disp,
                                  double* t_hi, double* t_lo, uint64_t* n_events, int32_t* status,
                                  akmc_stream stream);
/* Bytes of the concatenated species array, and number of vacancy slots. */
size_t akmc_batch_sites(const akmc_batch* batch);
int64_t akmc_batch_vacancies(const akmc_batch* batch);

/* Synchronise the stream and report voxel statuses: per_voxel (nullable,
 * n_voxels entries); returns AKMC_OK if every voxel is OK, else the status
 * of the lowest-indexed voxel that is not. */
akmc_status akmc_sync_status(akmc_batch* batch, akmc_stream stream, int32_t* per_voxel);

/* Workload proxy of the dynamic voxel scheduling (Sec. "Dynamic Voxel
 * Scheduling", Eq. 10: W_v ~ M_v exp(-E_v / (kB T_v)), M_v a multiplicity
 * of local events and E_v an effective barrier set by the voxel's defect
 * state), evaluated on the device from each voxel's current hop rates:
 *   M_hat[v] = number of admissible hops (rate > 0) of all its vacancies,
 *   W[v]     = Gamma_tot / nu (Gamma_tot = sum of its 8 n_vac hop rates),
 *   E_hat[v] = -kB T_v ln(W[v] / M_hat[v]) eV, the single barrier that gives
 *              every admissible hop the voxel's mean rate, so that
 *              W = M_hat exp(-E_hat / (kB T_v)) holds exactly (+inf if M_hat = 0).
 * Gamma_tot = nu W is the voxel's event rate: advancing it by dt of simulated
 * time takes about nu W dt events.  In pure Fe, E_hat = E0(Fe) and M_hat = 8
 * n_vac.  Outputs: host arrays of n_voxels doubles, each nullable.  Rebuilds
 * rates first after a state load; uses the batch's small I/O area, so it is
 * stream-ordered with the batch's other calls; synchronises the stream. */
akmc_status akmc_workload_proxy(akmc_batch* batch, double* W, double* M_hat, double* E_hat, akmc_stream stream);

/* Cu cluster size histogram of one voxel: connected components of Cu under
 * 1nn+2nn (mode 0) or 1nn (mode 1) adjacency; bins {1,2,3,4,5-9,10-19,
 * 20-49,>=50}.  Uses scratch memory inside the workspace; synchronises. */
akmc_status akmc_cluster_hist(akmc_batch* batch, int32_t voxel, int32_t mode,
                              int64_t hist[8], akmc_stream stream);

/* Allocation-free Cu cluster histogram (no counterpart in the paper).
 * For callers that cannot let a library allocate device memory: programs
 * whose GPU memory is owned entirely by another allocator (a framework or
 * simulation that reserves the device's memory up front and treats any
 * other cudaMalloc as an error or a source of fragmentation), and code on a
 * latency-critical path where an allocation could block or synchronise the
 * device.  Same result as akmc_cluster_hist on a lattice that is not part of
 * a batch: species is a device array of 2L^3 species codes (site order as
 * above), hist a device int64[8] that receives the bin counts (mode and bins
 * as akmc_cluster_hist).  The scratch (union-find labels and cluster sizes)
 * is a fixed file-scope device array of 2 x 524,288 int32 (4 MiB) that every
 * GPU which loads the library holds until the process exits; lattices above
 * 524,288 sites (L > 64) are rejected with AKMC_EINVAL.  The call allocates
 * nothing: no cudaMalloc, cudaFree or allocating library routine.  Its first
 * call on a device does a one-time set-up there (device addresses of the
 * static arrays and a copy of the neighbour tables into them, waited for
 * with a device synchronisation so that kernels on any stream see it), so
 * make that first call before any stream capture.  The set-up is not
 * repeated after cudaDeviceReset: do not call this entry point on a device
 * that was reset after its first call.  Every call shares the scratch
 * array, which keeps the last call's contents (each call re-initialises what
 * it needs); calls that overlap on the GPU -- on different streams, or from
 * different host threads -- race on it.  Stream-ordered; does not
 * synchronise. */
akmc_status akmc_cluster_hist_noalloc(const uint8_t* species, int32_t L, int32_t mode, int64_t* hist,
                                      akmc_stream stream);

/* Launch shape of akmc_step_n: warps per voxel-CTA (1, 2, 4, 8 or 16) and CTAs
 * per SM (0 = as many as fit).  Results are identical for every shape. */
akmc_status akmc_set_launch(akmc_batch* batch, int32_t warps_per_cta, int32_t ctas_per_sm);

int32_t akmc_n_voxels(const akmc_batch* batch);
void akmc_destroy_batch(akmc_batch* batch);      /* never frees caller memory */
const char* akmc_last_error(void);               /* thread-local, never NULL */

/* ---- global masked softmax sampling (logit form of the event selection) ----
 *
 * The action distribution of Eq. (1)-(2): every agent i of a system proposes
 * candidate transitions k with logits z_ik; admissible ones are scaled by 1/tau
 * (tau > 0), inadmissible ones are -inf, and one softmax over the concatenated
 * logits of all agents of the system selects one transition.  With
 * z = ln(Gamma) and tau = 1 this is the rejection-free selection (probability
 * Gamma / Gamma_tot).
 *
 * Input: one flat float32 device array of logits holding n_seg systems
 * ("segments") back to back; segment s covers [offsets[s], offsets[s+1]).
 * A logit is admissible iff mask[j] != 0 (mask: uint8 device array of the same
 * length, or NULL) and it is finite.  Segments may be empty and up to 2^30 long.
 *
 * Method (integer sums, so the draw does not depend on the launch shape): the
 * scaled logit is z * (1/tau) in FP32.  A segment is cut into parts of up to
 * 8192 logits; part p has maximum m_p and weights q_j = round(exp(z_j/tau -
 * m_p) 2^32) (FP32 exp) with exact int64 sum S_p.  With M = max m_p, the part
 * weights w_p = round(S_p exp(m_p - M)) (exactly S_p for a one-part segment);
 * u from Philox4x32-10 with key = seed and counter (counter_lo, counter_hi, s,
 * 0x53454c45); t = floor(u W), W = sum w_p; the part whose running sum of w
 * first exceeds t, then t - (the parts before) in the part's own units
 * (times S_p / w_p, rounded down), then the logit whose running sum of q first
 * exceeds that.
 *
 * akmc_select_scratch_bytes: device scratch needed for these offsets (host
 * array of n_seg+1 non-decreasing int64); 0 if the offsets are invalid.
 * akmc_select_plan: validates the offsets and writes the work plan into the
 * caller's scratch (256-byte aligned device memory, bytes >= the size above);
 * returns the number of parts in *n_parts; synchronises the stream.  The plan
 * stays valid for any number of akmc_select_logits calls with the same offsets.
 * akmc_select_logits: stream-ordered (two kernels, no host synchronisation,
 * capturable in a CUDA graph).  Outputs (device, n_seg entries): out_index[s] =
 * offset of the selected logit within segment s, or -1 if the segment has no
 * admissible logit; out_logp[s] = log of its probability (float32; NaN if none).
 * Errors: AKMC_EINVAL for NULL pointers, tau <= 0 or not finite, or n_seg /
 * n_parts that do not come from a plan; AKMC_ENOMEM if the scratch is too small.
 */
size_t akmc_select_scratch_bytes(const int64_t* host_offsets, int32_t n_seg);
akmc_status akmc_select_plan(const int64_t* host_offsets, int32_t n_seg, void* scratch, size_t bytes,
                             int32_t* n_parts, akmc_stream stream);
akmc_status akmc_select_logits(const float* logits, const uint8_t* mask, int32_t n_seg, int32_t n_parts, float tau,
                               uint64_t seed, uint64_t counter, const void* scratch, int64_t* out_index,
                               float* out_logp, akmc_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* AKMC_H */
