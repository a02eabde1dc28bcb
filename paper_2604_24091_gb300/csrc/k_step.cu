// k_step.cu -- the AKMC hot path: incremental rate refresh (a2-a5), event
// selection (a6), swap and density update (a7), refresh of affected vacancies
// (a8) and the compensated clock (a9), as one persistent kernel that steps a
// whole voxel per CTA, plus the full rebuild used by akmc_compute_rates.
//
// Design for GB300: a dependent float64 operation costs ~64 cycles there
// (float32: ~4.5), exp(double) ~1.1k and log(double) ~2.1k cycles, while an L2
// hit costs ~290.  The chain of one event is therefore kept off the FP64 pipe
// wherever the arithmetic allows:
//  * energies are exact integers (pair model: 2^-24 eV; EAM split precision:
//    2^-40 eV fixed point plus an FP32 polynomial part, rounded to 2^-24 eV);
//  * rates come from per-voxel tables of exp(-beta * Ea) on the 2^-25 eV grid
//    (two dependent FP64 multiplies instead of exp);
//  * selection compares non-negative doubles as integers (IEEE order);
//  * -ln(u2)/R of each event is batched and evaluated lane-parallel every
//    kClockBatch events, then folded into the compensated clock;
//  * the next event's Philox block is computed by an idle warp, with the
//    uniforms built from integers;
//  * the moved vacancy's read set is gathered before the event's density
//    updates (whose change it adds locally), so gathers never wait on atomics;
//  * hop terms are spread over all threads and summed as exact integers
//    (pair: 2^-24 eV; EAM split: 2^-40 eV), so the sums are order-free.
//
// One CTA owns one voxel at a time and runs all of its requested events; the
// voxel's rates, rate tree, tables and vacancy coordinates live in shared
// memory while it is resident.  Every result is independent of the launch
// shape: integer sums are order-free, and the FP64 mode rates hop k in one
// warp with a fixed lane mapping and shuffle tree.
#include <algorithm>
#include <mutex>

#include "akmc_device.cuh"
#include "akmc_launch.h"

namespace akmc {

constexpr int kClockBatch = 128;
constexpr long long kFBad = (long long)0x8000000000000000ull;   // window path: site embedding off the table

struct __align__(16) StepShared {
    double E0[4];
    double two_E0[4];
    double nu;
    double inv_knot;
    double phi_d[10][8];
    long long phi_q[10][8];
    const Cubic64* Fd;
    const float4* Ff;
    const long long* Fq;
    int32_t eps_q[2][25];
    int32_t fq[5][8];
    int32_t dkq[4][64];       // fq[A][sip] - fq[A][sim] at index sip + 8 sim (window path)
    long long dphi[10][64];   // phi_q[pi][sip] - phi_q[pi][sim] at index sip + 8 sim (window path)
    int32_t thr_hi[4], thr_lo[4];
    int32_t sph[64];
    int32_t off[160];
    uint32_t ent[8][80];
    int32_t mk[8];
    uint8_t dsh[160][8];
    // single-vacancy prefetch region (see phase_prefetch)
    uint16_t ridx[8][160];
    int32_t roff[288];
    int32_t rc[9];
    int32_t nreg;
    uint8_t rsp[288];
    int32_t rrho[288];
    int32_t n_rho, shift, cur_model, cur_small, vid;
    float inv_knot_f;
    VoxelDev v;
    uint64_t target;
    // staging of one vacancy's read set and its per-hop sums
    long long fsite[160];     // F_{s_u}(rho_u) of every read site (split mode, 2^-40 eV)
    int32_t srho[160];
    uint8_t ssp[160];
    uint8_t fbad[160];
    long long acc64[2][8];    // split mode: dE of each hop in 2^-40 eV (two partial sums)
    int32_t acc32[8];         // pair model: dE of each hop in 2^-24 eV
    double hop_de[8];         // FP64 mode
    int32_t hop_bad[8];
    // clock batch: u2 and R of each event, then dt in place of u2
    double cu2[kClockBatch];
    double cR[kClockBatch];
    double t_hi, t_lo;
    double nu1, nu2;      // uniforms of the next event
    uint64_t n;
    int32_t ccount;
    int32_t stop, numeric, n_aff;
    int32_t slot, dir, A;
    int32_t wX, wY, wZ, mX, mY, mZ;
    // single-vacancy lattice window (see run_events_window)
    int32_t W, ox, oy, oz;            // edge and origin (cells) of the window
    int32_t lX, lY, lZ, wb;           // vacancy: local half-unit coordinates, window index
    int32_t recenter;
    int32_t hsp[8], hbad[2][8];       // hop atoms and range flags from the terms phase
    int32_t pA, pw, pm, pwb, pmb;     // hop whose density change is pending: atom, window sites, parities
    int32_t pwX, pwY, pwZ, pmX, pmY, pmZ;
    double nx1, nx2;                  // uniforms of the event after the next one
    uint64_t nuU1, nxU1;              // u1 of the next / following event as a 53-bit integer (u1 = U1 2^-53)
    // sublattice superstep (see sl_kernel): counter words of the uniforms,
    // octant bounds (cells) and the octant's clock and window
    int32_t sl_on, sl_k, sl_sid, sl_n, sl_nvtot, sl_etab;
    int32_t* sl_stale;                // per vacancy: stored rates out of date (global)
    int32_t wrot;                     // window path: rotation of the warp roles (threads)
    int32_t sl_x0, sl_y0, sl_z0, sl_h;
    double sl_t, sl_T;
};

// Staging of one vacancy's read set and hop sums, for the general path's
// refresh of several vacancies per pass (kG at a time).
constexpr int kG = 4;
struct __align__(16) Grp {
    long long fsite[kEamU];   // split precision: F_{s_u}(rho_u) in 2^-40 eV
    int32_t srho[kEamU];
    long long acc64[2][8];
    double hop_de[8];
    int32_t acc32[8];
    int32_t hop_bad[8];
    uint8_t ssp[kEamU];
    uint8_t fbad[kEamU];
};

struct Dyn {
    double* tree;
    double* rates;
    double* dE;
    double* hsum;     // per vacancy: [1] vacancy sum, [2..3] half sums, [4..7] pair sums
    double* etab;
    int32_t* pos;
    int32_t* X;
    int32_t* Y;
    int32_t* Z;
    int32_t* disp;
    int32_t* aff;
    uint8_t* hop_sp;
    uint8_t* wsp;     // window species (single-vacancy path; padded layout, see widx)
    int32_t* wrho;    // window densities (same layout)
    int32_t* dprev;   // window path: density change of the last hop, [8 dirs][4 atoms][145 read-set sites]
    int32_t* gslot;   // sublattice superstep: voxel slot of each local vacancy
    int32_t* on;      // sublattice superstep: local vacancy still in the active octant
    int32_t* apos;    // sublattice superstep: packed half-unit coordinates of every vacancy at the start
    int32_t* lmap;    // sublattice superstep: local index of every vacancy, -1 if not local
    int32_t* fr;      // sublattice superstep: local vacancy's stored rates are current
    Grp* grp;         // general path with several vacancies: kG staging blocks
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Offsets of the dynamic shared-memory arrays (16-byte aligned).
struct DynLayout {
    size_t off[21];
    size_t total;
};

__host__ __device__ inline int win_sites(int W);

__host__ __device__ inline DynLayout dyn_layout(int max_nv, int max_P, int win) {
    const size_t nw = win > 0 ? (size_t)win_sites(win) : 0;
    const size_t sz[21] = {sizeof(double) * 2 * max_P, sizeof(double) * 8 * max_nv,
                           sizeof(double) * 8 * max_nv, sizeof(double) * 8 * max_nv,
                           sizeof(double) * kEtab,      sizeof(int32_t) * max_nv,
                           sizeof(int32_t) * max_nv,    sizeof(int32_t) * max_nv,
                           sizeof(int32_t) * max_nv,    sizeof(int32_t) * 3 * max_nv,
                           sizeof(int32_t) * max_nv,    (size_t)8 * max_nv,
                           nw,                          sizeof(int32_t) * nw,
                           win > 0 ? sizeof(int32_t) * kEamU * 32 : 0,
                           sizeof(int32_t) * max_nv,    sizeof(int32_t) * max_nv,
                           sizeof(int32_t) * max_nv,    sizeof(int32_t) * max_nv,
                           sizeof(int32_t) * max_nv,    max_nv > 1 ? sizeof(Grp) * kG : 0};
    DynLayout l;
    size_t o = 0;
    for (int i = 0; i < 21; ++i) {
        l.off[i] = o;
        o = align16(o + sz[i]);
    }
    l.total = o;
    return l;
}

__device__ __forceinline__ Dyn carve(unsigned char* base, int max_nv, int max_P, int win) {
    const DynLayout l = dyn_layout(max_nv, max_P, win);
    Dyn d;
    d.tree = (double*)(base + l.off[0]);
    d.rates = (double*)(base + l.off[1]);
    d.dE = (double*)(base + l.off[2]);
    d.hsum = (double*)(base + l.off[3]);
    d.etab = (double*)(base + l.off[4]);
    d.pos = (int32_t*)(base + l.off[5]);
    d.X = (int32_t*)(base + l.off[6]);
    d.Y = (int32_t*)(base + l.off[7]);
    d.Z = (int32_t*)(base + l.off[8]);
    d.disp = (int32_t*)(base + l.off[9]);
    d.aff = (int32_t*)(base + l.off[10]);
    d.hop_sp = (uint8_t*)(base + l.off[11]);
    d.wsp = win > 0 ? (uint8_t*)(base + l.off[12]) : nullptr;
    d.wrho = win > 0 ? (int32_t*)(base + l.off[13]) : nullptr;
    d.dprev = win > 0 ? (int32_t*)(base + l.off[14]) : nullptr;
    d.gslot = (int32_t*)(base + l.off[15]);
    d.on = (int32_t*)(base + l.off[16]);
    d.apos = (int32_t*)(base + l.off[17]);
    d.lmap = (int32_t*)(base + l.off[18]);
    d.fr = (int32_t*)(base + l.off[19]);
    d.grp = max_nv > 1 ? (Grp*)(base + l.off[20]) : nullptr;
    return d;
}

size_t step_dyn_smem(int max_nv, int max_P, int win) { return dyn_layout(max_nv, max_P, win).total; }


// Order of non-negative doubles equals the order of their bit patterns.
__device__ __forceinline__ bool lt_nonneg(double a, double b) {
    return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ bool is_zero(double a) { return __double_as_longlong(a) == 0; }

template <int NW>
__device__ void load_model(StepShared& S, const ModelDev* M) {
    const int tid = threadIdx.x;
    for (int i = tid; i < 50; i += NW * 32) S.eps_q[i / 25][i % 25] = M->eps_q[i / 25][i % 25];
    for (int i = tid; i < 40; i += NW * 32) S.fq[i / 8][i % 8] = M->fq[i / 8][i % 8];
    for (int i = tid; i < 80; i += NW * 32) {
        S.phi_d[i / 8][i % 8] = M->phi_d[i / 8][i % 8];
        S.phi_q[i / 8][i % 8] = M->phi_q[i / 8][i % 8];
    }
    for (int i = tid; i < 4 * 64; i += NW * 32) {
        const int A = i >> 6, sp = i & 7, sm = (i >> 3) & 7;
        S.dkq[A][i & 63] = M->fq[A][sp] - M->fq[A][sm];
    }
    for (int i = tid; i < 10 * 64; i += NW * 32) {
        const int pi = i >> 6, sp = i & 7, sm = (i >> 3) & 7;
        S.dphi[pi][i & 63] = M->phi_q[pi][sp] - M->phi_q[pi][sm];
    }
    if (tid < 4) {
        S.E0[tid] = M->E0[tid];
        S.two_E0[tid] = M->two_E0[tid];
        S.thr_hi[tid] = M->thr_hi[tid];
        S.thr_lo[tid] = M->thr_lo[tid];
    }
    if (tid == 0) {
        S.nu = M->nu;
        S.Fd = M->Fd;
        S.Ff = M->Ff;
        S.Fq = M->Fq;
        S.n_rho = M->n_rho;
        S.shift = M->shift;
        S.inv_knot = M->inv_knot;
        S.inv_knot_f = (float)M->inv_knot;
        S.cur_model = -1;
        S.cur_small = -1;
        S.sl_on = 0;
    }
}

// Stencil tables of the voxel's energy model (reloaded only when the model or
// the L = 4 special case changes).
template <int NW>
__device__ void load_tables(StepShared& S, const Tables* T, int model, int small) {
    const int tid = threadIdx.x;
    if (S.cur_model == model && S.cur_small == small) return;   // uniform: read after a barrier
    __syncthreads();
    if (model == 0) {
        for (int i = tid; i < 64; i += NW * 32) S.off[i] = T->pair_off[i];
        for (int i = tid; i < 8 * 32; i += NW * 32) S.ent[i / 32][i % 32] = T->pair_ent[i / 32][i % 32];
        if (tid < 8) S.mk[tid] = T->pair_mk[tid];
        for (int i = tid; i < 160; i += NW * 32) S.roff[i] = T->pair_roff[i];
        for (int i = tid; i < 8 * 64; i += NW * 32) S.ridx[i / 64][i % 64] = T->pair_ridx[i / 64][i % 64];
        if (tid < 9) S.rc[tid] = T->pair_rc[tid];
        if (tid == 0) S.nreg = T->pair_nreg;
    } else {
        for (int i = tid; i < 160; i += NW * 32) S.off[i] = T->eam_off[i];
        for (int i = tid; i < 8 * 80; i += NW * 32) S.ent[i / 80][i % 80] = T->eam_ent[i / 80][i % 80];
        if (tid < 8) S.mk[tid] = T->eam_mk[tid];
        for (int i = tid; i < 64; i += NW * 32) S.sph[i] = T->sph_off[i];
        for (int i = tid; i < 160 * 8; i += NW * 32) S.dsh[i / 8][i % 8] = T->eam_dsh[small][i / 8][i % 8];
        for (int i = tid; i < 288; i += NW * 32) S.roff[i] = T->eam_roff[i];
        for (int i = tid; i < 8 * 160; i += NW * 32) S.ridx[i / 160][i % 160] = T->eam_ridx[i / 160][i % 160];
        if (tid < 9) S.rc[tid] = T->eam_rc[tid];
        if (tid == 0) S.nreg = T->eam_nreg;
    }
    __syncthreads();
    if (tid == 0) {
        S.cur_model = model;
        S.cur_small = small;
    }
    __syncthreads();
}

// Embedding function on the fixed-point density r (split precision): knot
// k = r >> shift, t = (r - k 2^shift) 2^-shift, built exactly from the bits of
// the remainder.  The knot value is exact in 2^-40 eV; the Hermite part
// t (c1 + t (c2 + t c3)) is evaluated in FP32 (|part| < 0.5 eV) and rounded to
// 2^-40 eV; the result is one integer in units of 2^-40 eV.  The coefficient
// table has a zero entry at the last knot, so r = (n_rho - 1) 2^shift gives the
// last knot value exactly; r outside [0, (n_rho - 1) 2^shift] is clamped to it
// and flagged.
struct EmbedC {
    const float4* Ff;
    const long long* Fq;
    int n_rho, shift;
    unsigned lim;      // (n_rho - 1) << shift
};

__device__ __forceinline__ long long embed_c(const EmbedC& E, int a, int r, int& bad) {
    const unsigned ur = (unsigned)r;
    bad |= ur > E.lim;
    const unsigned k = min(ur >> E.shift, (unsigned)(E.n_rho - 1));
    const float t = __int_as_float(0x3F800000 | ((ur & ((1u << E.shift) - 1u)) << (23 - E.shift))) - 1.0f;
    const int i = a * E.n_rho + (int)k;
    const float4 c = __ldg(&E.Ff[i]);
    const float p = t * (c.x + t * (c.y + t * c.z));
    return __ldg(&E.Fq[i]) + __float2ll_rn(p * 1099511627776.0f);
}

__device__ __forceinline__ EmbedC embed_consts(const StepShared& S) {
    EmbedC E;
    E.Ff = S.Ff;
    E.Fq = S.Fq;
    E.n_rho = S.n_rho;
    E.shift = S.shift;
    E.lim = (unsigned)(S.n_rho - 1) << S.shift;
    return E;
}

__device__ __forceinline__ long long embed_q(const StepShared& S, int a, int r, int& bad) {
    return embed_c(embed_consts(S), a, r, bad);
}

__device__ __forceinline__ double embed_fp64(const StepShared& S, int a, int r, int& bad) {
    const int last = S.n_rho - 1;
    int k = r >> S.shift;
    if (r < 0 || k > last || (k == last && (r & ((1 << S.shift) - 1)))) bad = 1;
    k = min(max(k, 0), last - 1);
    double t = (double)(r - (k << S.shift)) * S.inv_knot;
    const Cubic64& c = S.Fd[a * last + k];
    return c.F + t * (c.c1 + t * (c.c2 + t * c.c3));
}

// (a4) Barrier Ea = max(0, dE, E0[A] + dE/2) and rate nu * exp(-beta Ea) of one
// hop.  With y = dE/2 + 2 (middle branch, constant K = nu exp(beta (2 - E0))) or
// y = dE (Ea = dE branch, K = nu), rate = K exp(-beta y); for 0 <= y < 4 eV,
// exp(-beta y) is the product of three table entries indexed by the 27 bits of
// y * 2^25 (times a 3rd-order correction for a float64 dE that is not on the
// grid).  Other y, or tables that over/underflow, use exp directly.
// On the grid (dE = q 2^-24 eV) the branch choice and indexing are integer
// selects, so the 8 lanes do not diverge.
__device__ __forceinline__ double hop_rate_grid(const StepShared& S, const Dyn& D, int A, int q) {
    const int Ai = A < 4 ? A : 3;
    if (!S.v.etab_ok) {
        const double de = (double)q * 0x1p-24;
        const double Ea = fmax(fmax(0.0, de), S.E0[Ai] + 0.5 * de);
        return A == kVac ? 0.0 : S.nu * exp(-(Ea * S.v.beta));
    }
    const bool zero = q < S.thr_lo[Ai], up = q > S.thr_hi[Ai];
    const long long j = zero ? 0 : (up ? 2LL * q : (long long)q + (1LL << 26));
    const double K = (zero || up) ? S.nu : D.etab[1536 + Ai];
    double g;
    if (j >= 0 && j < (1LL << 27)) {
        const int ji = (int)j;
        g = (K * D.etab[ji & 511]) * (D.etab[512 + ((ji >> 9) & 511)] * D.etab[1024 + (ji >> 18)]);
    } else {
        g = K * exp(-(S.v.beta * ((double)j * 0x1p-25)));
    }
    return A == kVac ? 0.0 : g;
}

__device__ __forceinline__ double hop_rate_fp64(const StepShared& S, const Dyn& D, int A, double de) {
    if (A == kVac) return 0.0;
    if (!S.v.etab_ok) {
        const double Ea = fmax(fmax(0.0, de), S.E0[A] + 0.5 * de);
        return S.nu * exp(-(Ea * S.v.beta));
    }
    if (de < -S.two_E0[A]) return S.nu;
    double K, y;
    if (de > S.two_E0[A]) { K = S.nu; y = de; } else { K = D.etab[1536 + A]; y = fma(de, 0.5, 2.0); }
    const double yj = y * 0x1p25;
    if (!(yj >= 0.0 && yj < 134217728.0)) return K * exp(-(S.v.beta * y));
    const int j = (int)yj;
    const double r = fma(-(double)j, 0x1p-25, y);
    const double x = S.v.beta * r;
    const double corr = fma(fma(fma(-x, 0.16666666666666666, 0.5), x, -1.0), x, 1.0);
    return (K * D.etab[j & 511]) * ((D.etab[512 + ((j >> 9) & 511)] * D.etab[1024 + (j >> 18)]) * corr);
}

__device__ __forceinline__ bool finite_bits(double g) {
    return ((__double_as_longlong(g) >> 52) & 0x7ff) != 0x7ff;
}

// A non-negative float64 x as an unsigned fixed-point mantissa M in
// [2^63, 2^64) and a binary exponent E, x = M 2^E (M = 0 for zero and
// subnormal x).
__device__ __forceinline__ void rate_to_fixed(double x, unsigned long long& M, int& E) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int be = (int)((b >> 52) & 0x7ff);
    M = be == 0 ? 0ull : (((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11);
    E = be - 1075 - 11;
}

// (a4) hop_rate_grid's rate as M 2^E with M in [2^60, 2^64): the same table
// entries, their 53-bit mantissas multiplied in integers (three 64 x 64-bit
// products, each truncated to its upper 64 bits; relative error below 2^-59),
// so the selection needs no float64 arithmetic.  Where hop_rate_grid calls
// exp (tables unusable, or the energy off their range) the float64 rate is
// converted instead; a non-finite rate sets bad.
__device__ __forceinline__ void hop_rate_fixed(const StepShared& S, const Dyn& D, int A, int q, bool etab_ok,
                                               unsigned long long& M, int& E, int& bad) {
    if (A == kVac) {
        M = 0;
        E = 0;
        return;
    }
    const int Ai = A < 4 ? A : 3;
    const bool zero = q < S.thr_lo[Ai], up = q > S.thr_hi[Ai];
    const long long j = zero ? 0 : (up ? 2LL * q : (long long)q + (1LL << 26));
    if (!etab_ok || !(j >= 0 && j < (1LL << 27))) {
        const double g = hop_rate_grid(S, D, A, q);
        bad |= !finite_bits(g);
        rate_to_fixed(g, M, E);
        return;
    }
    const int ji = (int)j;
    const unsigned long long bK = (unsigned long long)__double_as_longlong((zero || up) ? S.nu : D.etab[1536 + Ai]);
    const unsigned long long b0 = (unsigned long long)__double_as_longlong(D.etab[ji & 511]);
    const unsigned long long b1 = (unsigned long long)__double_as_longlong(D.etab[512 + ((ji >> 9) & 511)]);
    const unsigned long long b2 = (unsigned long long)__double_as_longlong(D.etab[1024 + (ji >> 18)]);
    auto m11 = [](unsigned long long b) { return ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11; };
    auto ex = [](unsigned long long b) { return (int)((b >> 52) & 0x7ff) - 1075; };
    const unsigned long long a = __umul64hi(m11(bK), m11(b0));   // floor(mK m0 / 2^42) in [2^62, 2^64)
    const unsigned long long c = __umul64hi(m11(b1), m11(b2));   // floor(m1 m2 / 2^42)
    M = __umul64hi(a, c);                                        // floor(a c / 2^64) in [2^60, 2^64)
    E = ex(bK) + ex(b0) + ex(b1) + ex(b2) + 148;
}

// Uniforms of event n built from the Philox block with integer operations
// (exact: a 53-bit integer times 2^-53).
__device__ __forceinline__ double u53_to_double(uint64_t a) {
    if (a == 0) return 0.0;
    const int e = 63 - __clzll((long long)a);           // top bit position, <= 53
    const uint64_t mant = (a << (52 - e)) & 0xFFFFFFFFFFFFFull;
    return __longlong_as_double((long long)(((uint64_t)(e - 53 + 1023) << 52) | mant));
}

// Regular events: counter (n_lo, n_hi, uid_lo, uid_hi & 0x7fffffff).  Event i of
// a sublattice superstep k in sector c: counter (i, k, c, 0xC0000000 | uid_lo
// & 0x3fffffff) -- the top bits keep the two families of counters disjoint.
__device__ __forceinline__ void next_uniforms(StepShared& S) {
    const uint64_t n = S.n, uid = S.v.uid, seed = S.v.seed;
    uint32_t c0 = (uint32_t)n, c1 = (uint32_t)(n >> 32), c2 = (uint32_t)uid,
             c3 = (uint32_t)(uid >> 32) & 0x7fffffffu;
    if (S.sl_on) {
        c1 = (uint32_t)S.sl_k;
        c2 = (uint32_t)S.sl_sid;
        c3 = 0xC0000000u | ((uint32_t)uid & 0x3FFFFFFFu);
    }
    philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    S.nuU1 = ((uint64_t)c0 << 21) | (c1 >> 11);
    S.nu1 = u53_to_double(S.nuU1);
    S.nu2 = u53_to_double((((uint64_t)c2 << 21) | (c3 >> 11)) + 1);
}

// ---- (a2)-(a5): rates of the 8 hops of one vacancy, in phases ----------------
// G  gather the read set (all threads);
// F  split precision: embedding value of every read site (all threads);
// E  hop energy changes (all threads) and, for the vacancy that just moved,
//    this event's density updates (a7);
// R  rates, subtree sums and tree path (lanes 0..7 of warp 0).
// A barrier separates G, F, E and R.  For the vacancy that just moved (w ->
// m) the read set is gathered before this event's density updates reach
// memory and the hop's density change is added locally.

template <int NW, int MODE>
__device__ __forceinline__ void phase_gather(StepShared& S, const Dyn& D, int q, bool moved) {
    constexpr int NT = NW * 32;
    constexpr bool eam = MODE != 0;
    constexpr int U = eam ? kEamU : kPairU;
    const int tid = threadIdx.x;
    const int L = S.v.L, M2 = 2 * L;
    const int X = D.X[q], Y = D.Y[q], Z = D.Z[q];
    if (moved && tid == NT - 1) next_uniforms(S);   // the next event's Philox block, off the critical path
    for (int u = tid; u < U; u += NT) {
        const int o = S.off[u];
        const int s = site_index(wrap_coord(X + off_dx(o), M2), wrap_coord(Y + off_dy(o), M2),
                                 wrap_coord(Z + off_dz(o), M2), L);
        S.ssp[u] = S.sl_on ? __ldcg(S.v.species + s) : S.v.species[s];
        if (eam) {
            int r = S.sl_on ? __ldcg(S.v.rho + s) : S.v.rho[s];
            if (moved) {
                const int ds = S.dsh[u][S.dir];
                r += S.fq[S.A][ds >> 3] - S.fq[S.A][ds & 7];
            }
            S.srho[u] = r;
        }
    }
    if (tid < 16) S.acc64[tid >> 3][tid & 7] = 0;
    if (tid < 8) {
        S.acc32[tid] = 0;
        S.hop_bad[tid] = 0;
    }
}

// Single-vacancy fast path.  phase_prefetch loads the region around the
// vacancy's current position (the read sets of all 8 possible next
// positions) into shared memory; it runs in the shadow of warp 0's rate
// phase, after the event's density updates are visible.  phase_fill then
// builds the next event's read set from that region instead of memory: the
// swapped sites take their new species, and every density gets the hop's
// change added.  Needs no periodic aliasing inside the region (L >= 6 for
// EAM, L >= 5 for the pair model).
template <int NW, int MODE>
__device__ __forceinline__ void phase_prefetch(StepShared& S, const Dyn& D, int first_tid) {
    constexpr int NT = NW * 32;
    const int i0 = (int)threadIdx.x - first_tid;
    if (i0 < 0) return;
    const int L = S.v.L, M2 = 2 * L;
    const int X = D.X[0], Y = D.Y[0], Z = D.Z[0];
    for (int i = i0; i < S.nreg; i += NT - first_tid) {
        const int o = S.roff[i];
        const int s = site_index(wrap_coord(X + off_dx(o), M2), wrap_coord(Y + off_dy(o), M2),
                                 wrap_coord(Z + off_dz(o), M2), L);
        S.rsp[i] = S.sl_on ? __ldcg(S.v.species + s) : S.v.species[s];
        if (MODE != 0) S.rrho[i] = S.sl_on ? __ldcg(S.v.rho + s) : S.v.rho[s];
    }
}

template <int NW, int MODE>
__device__ __forceinline__ void phase_fill(StepShared& S) {
    constexpr int NT = NW * 32;
    constexpr int U = MODE != 0 ? kEamU : kPairU;
    const int tid = threadIdx.x;
    const int d = S.dir, A = S.A;
    const int rc_old = S.rc[8], rc_new = S.rc[d];
    if (tid == NT - 1) next_uniforms(S);   // the next event's Philox block
    for (int u = tid; u < U; u += NT) {
        const int ri = S.ridx[d][u];
        const int sp = ri == rc_old ? A : (ri == rc_new ? kVac : S.rsp[ri]);
        S.ssp[u] = (uint8_t)sp;
        if (MODE != 0) {
            const int ds = S.dsh[u][d];
            const int r = S.rrho[ri] + S.fq[A][ds >> 3] - S.fq[A][ds & 7];
            S.srho[u] = r;
            if (MODE == 1) {
                int bad = 0;
                S.fsite[u] = sp == kVac ? 0 : embed_q(S, sp, r, bad);
                S.fbad[u] = (uint8_t)bad;
            }
        }
    }
    if (tid < 16) S.acc64[tid >> 3][tid & 7] = 0;
    if (tid < 8) {
        S.acc32[tid] = 0;
        S.hop_bad[tid] = 0;
    }
}

template <int NW>
__device__ __forceinline__ void phase_site_embed(StepShared& S) {
    for (int u = threadIdx.x; u < kEamU; u += NW * 32) {
        const int a = S.ssp[u];
        int bad = 0;
        S.fsite[u] = a == kVac ? 0 : embed_q(S, a, S.srho[u], bad);
        S.fbad[u] = (uint8_t)bad;
    }
}

template <int NW, int MODE>
__device__ __forceinline__ void phase_terms(StepShared& S, bool moved) {
    constexpr int NT = NW * 32;
    constexpr bool eam = MODE != 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (MODE == 0) {
        // (a2) dE = sum over the 13 bonds of w (V -> A) and 13 bonds of m (A -> V),
        // exact integers in units of 2^-24 eV (order-free accumulation).
        for (int it = tid; it < 8 * kPairE; it += NT) {
            const int k = it / kPairE, e = it - k * kPairE;
            const int A = S.ssp[S.mk[k]];
            if (A == kVac) continue;
            const uint32_t en = S.ent[k][e];
            const int x = S.ssp[en & 0xff], sh = (en >> 8) & 1;
            const int t = S.eps_q[sh][A * 5 + x] - S.eps_q[sh][kVac * 5 + x];
            atomicAdd(&S.acc32[k], (en >> 9) & 1 ? -t : t);
        }
    } else if (MODE == 1) {
        // (a3) dE = sum_i [F(rho_i + drho_i) - F(rho_i)] + own term + pair terms,
        // every term an integer in 2^-40 eV; one (or two) warps per hop, integer
        // shuffle sums.
        constexpr int WPH = NW >= 16 ? 2 : 1;
        for (int kk = warp; kk < 8 * WPH; kk += NW) {
            const int k = kk & 7, half = kk >> 3;
            const int A = S.ssp[S.mk[k]];
            if (A == kVac) continue;
            long long v = 0;
            int bad = 0;
            for (int e = half * 32 + lane; e < kEamE; e += 32 * WPH) {
                const uint32_t en = S.ent[k][e];
                if (en >> 14) {
                    const int mk = S.mk[k];
                    v += embed_q(S, A, S.srho[0] - S.fq[A][1], bad) - S.fsite[mk];
                    bad |= S.fbad[mk];
                } else {
                    const int idx = en & 0xff, sip = (en >> 8) & 7, sim = (en >> 11) & 7;
                    const int a = S.ssp[idx];
                    if (a == kVac) continue;
                    const int pi = pair_index(A, a);
                    v += embed_q(S, a, S.srho[idx] + S.fq[A][sip] - S.fq[A][sim], bad) - S.fsite[idx] +
                         (S.phi_q[pi][sip] - S.phi_q[pi][sim]);
                    bad |= S.fbad[idx];
                }
            }
            v = warp_sum(v);
            bad = __any_sync(0xffffffffu, bad);
            if (lane == 0) {
                S.acc64[half][k] = v;
                if (bad) S.hop_bad[k] = 1;
            }
        }
    } else {
        // (a3) FP64 throughout: one warp per hop, fixed lane order and shuffle tree.
        for (int k = warp; k < 8; k += NW) {
            const int A = S.ssp[S.mk[k]];
            if (A == kVac) {
                if (lane == 0) S.hop_de[k] = 0.0;
                continue;
            }
            double acc = 0.0;
            int bad = 0;
            for (int j = lane; j < kEamE; j += 32) {
                const uint32_t en = S.ent[k][j];
                int a, r0, r1;
                double ph = 0.0;
                if (en >> 14) {
                    a = A;
                    r0 = S.srho[S.mk[k]];
                    r1 = S.srho[0] - S.fq[A][1];
                } else {
                    const int idx = en & 0xff, sip = (en >> 8) & 7, sim = (en >> 11) & 7;
                    a = S.ssp[idx];
                    if (a == kVac) continue;
                    r0 = S.srho[idx];
                    r1 = r0 + S.fq[A][sip] - S.fq[A][sim];
                    const int pi = pair_index(A, a);
                    ph = S.phi_d[pi][sip] - S.phi_d[pi][sim];
                }
                acc += (embed_fp64(S, a, r1, bad) - embed_fp64(S, a, r0, bad)) + ph;
            }
            acc = warp_sum(acc);
            bad = __any_sync(0xffffffffu, bad);
            if (lane == 0) {
                S.hop_de[k] = acc;
                S.hop_bad[k] = bad;
            }
        }
    }
    // (a7) this event's density updates, now that the read set is in shared memory:
    // rho_i += f_A(r_iw) over S(w), -= f_A(r_im) over S(m).
    if (eam && moved) {
        const int L = S.v.L, M2 = 2 * L;
        for (int i = tid; i < 2 * kSph; i += NT) {
            const int side = i >= kSph;
            const int o = S.sph[side ? i - kSph : i];
            const int cX = side ? S.mX : S.wX, cY = side ? S.mY : S.wY, cZ = side ? S.mZ : S.wZ;
            const int s = site_index(wrap_coord(cX + off_dx(o), M2), wrap_coord(cY + off_dy(o), M2),
                                     wrap_coord(cZ + off_dz(o), M2), L);
            const int f = S.fq[S.A][off_extra(o)];
            atomicAdd(&S.v.rho[s], side ? -f : f);
        }
    }
}

// R: (a4) rates of the 8 hops in lanes 0..7 of warp 0; (a5) subtree sums
// (g0+g1), (g2+g3), ..., ((g0+g1)+(g2+g3)), ((g4+g5)+(g6+g7)), the vacancy sum
// and its tree path.  Only warp 0 executes this; it ends with __syncwarp.
template <int MODE>
__device__ __forceinline__ void phase_rates(StepShared& S, const Dyn& D, int q) {
    const int lane = threadIdx.x & 31;
    if (lane < 8) {
        const int A = S.ssp[S.mk[lane]];
        double de, g;
        if (MODE == 2) {
            de = S.hop_de[lane];
            g = hop_rate_fp64(S, D, A, de);
        } else {
            const int dq = MODE == 0 ? S.acc32[lane]
                                     : (int)((S.acc64[0][lane] + S.acc64[1][lane] + (1LL << 15)) >> 16);
            de = A == kVac ? 0.0 : (double)dq * 0x1p-24;
            g = hop_rate_grid(S, D, A, dq);
        }
        int bad = S.hop_bad[lane] | !finite_bits(g);
        const double s1 = g + __shfl_xor_sync(0xffu, g, 1);
        const double s2 = s1 + __shfl_xor_sync(0xffu, s1, 2);
        const double s3 = s2 + __shfl_xor_sync(0xffu, s2, 4);
        bad = __any_sync(0xffu, bad);
        D.rates[8 * q + lane] = g;
        D.dE[8 * q + lane] = de;
        D.hop_sp[8 * q + lane] = (uint8_t)A;
        double* h = D.hsum + 8 * q;
        if ((lane & 1) == 0) h[4 + (lane >> 1)] = s1;
        if ((lane & 3) == 0) h[2 + (lane >> 2)] = s2;
        if (lane == 0) {
            h[1] = s3;
            const int P = S.v.P;
            D.tree[P + q] = s3;
            for (int i = (P + q) >> 1; i >= 1; i >>= 1) D.tree[i] = D.tree[2 * i] + D.tree[2 * i + 1];
            if (bad) S.numeric = 1;
        }
    }
    __syncwarp();
}

// ---- general path, several vacancies per pass --------------------------------
// After a hop the rates of the moved vacancy and of every vacancy within reach
// of it are recomputed together, kG vacancies per pass: the read sets are
// gathered from memory (the hop's density updates are already there), then
// site embeddings, hop terms and rates run over all of them at once, so a pass
// costs the barriers of one vacancy whatever the number refreshed.  The
// arithmetic of every vacancy is that of the one-vacancy phases above.

// (a7) the hop's density updates (rho_i += f_A(r_iw) over S(w), -= f_A(r_im)
// over S(m)) and the list of other vacancies whose read set may contain a
// changed site (every vacancy within `reach` half units of w per axis).
template <int NW, int MODE>
__device__ __forceinline__ void phase_hop_update(StepShared& S, const Dyn& D) {
    constexpr int NT = NW * 32;
    constexpr int reach = MODE != 0 ? 8 : 4;
    const int tid = threadIdx.x;
    const int L = S.v.L, M2 = 2 * L;
    if (tid == NT - 1) next_uniforms(S);   // the next event's Philox block
    if (MODE != 0) {
        for (int i = tid; i < 2 * kSph; i += NT) {
            const int side = i >= kSph;
            const int o = S.sph[side ? i - kSph : i];
            const int cX = side ? S.mX : S.wX, cY = side ? S.mY : S.wY, cZ = side ? S.mZ : S.wZ;
            const int s = site_index(wrap_coord(cX + off_dx(o), M2), wrap_coord(cY + off_dy(o), M2),
                                     wrap_coord(cZ + off_dz(o), M2), L);
            const int f = S.fq[S.A][off_extra(o)];
            atomicAdd(&S.v.rho[s], side ? -f : f);
        }
    }
    for (int q = tid; q < S.v.nv; q += NT) {
        if (q == S.slot) continue;
        int ddx = D.X[q] - S.wX, ddy = D.Y[q] - S.wY, ddz = D.Z[q] - S.wZ;
        ddx = ddx >= L ? ddx - M2 : (ddx < -L ? ddx + M2 : ddx);
        ddy = ddy >= L ? ddy - M2 : (ddy < -L ? ddy + M2 : ddy);
        ddz = ddz >= L ? ddz - M2 : (ddz < -L ? ddz + M2 : ddz);
        if (abs(ddx) <= reach && abs(ddy) <= reach && abs(ddz) <= reach) D.aff[atomicAdd(&S.n_aff, 1)] = q;
    }
}

// vacancy of entry g0 + g of the refresh list: the moved one first
__device__ __forceinline__ int grp_vacancy(const StepShared& S, const Dyn& D, int i) {
    return i == 0 ? S.slot : D.aff[i - 1];
}

template <int NW, int MODE>
__device__ __forceinline__ void grp_gather(StepShared& S, const Dyn& D, int g0, int n) {
    constexpr int NT = NW * 32;
    constexpr int U = MODE != 0 ? kEamU : kPairU;
    const int tid = threadIdx.x;
    const int L = S.v.L, M2 = 2 * L;
    for (int i = tid; i < n * U; i += NT) {
        const int g = i / U, u = i - g * U;
        const int q = grp_vacancy(S, D, g0 + g);
        const int o = S.off[u];
        const int s = site_index(wrap_coord(D.X[q] + off_dx(o), M2), wrap_coord(D.Y[q] + off_dy(o), M2),
                                 wrap_coord(D.Z[q] + off_dz(o), M2), L);
        Grp& G = D.grp[g];
        G.ssp[u] = S.v.species[s];
        if (MODE != 0) G.srho[u] = S.v.rho[s];
    }
    for (int i = tid; i < n * 8; i += NT) {
        Grp& G = D.grp[i >> 3];
        G.acc64[0][i & 7] = 0;
        G.acc64[1][i & 7] = 0;
        G.acc32[i & 7] = 0;
        G.hop_bad[i & 7] = 0;
    }
}

template <int NW>
__device__ __forceinline__ void grp_site_embed(StepShared& S, const Dyn& D, int n) {
    for (int i = threadIdx.x; i < n * kEamU; i += NW * 32) {
        const int g = i / kEamU, u = i - g * kEamU;
        Grp& G = D.grp[g];
        const int a = G.ssp[u];
        int bad = 0;
        G.fsite[u] = a == kVac ? 0 : embed_q(S, a, G.srho[u], bad);
        G.fbad[u] = (uint8_t)bad;
    }
}

template <int NW, int MODE>
__device__ __forceinline__ void grp_terms(StepShared& S, const Dyn& D, int n) {
    constexpr int NT = NW * 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (MODE == 0) {
        for (int it = tid; it < n * 8 * kPairE; it += NT) {
            const int g = it / (8 * kPairE), r = it - g * 8 * kPairE, k = r / kPairE, e = r - k * kPairE;
            Grp& G = D.grp[g];
            const int A = G.ssp[S.mk[k]];
            if (A == kVac) continue;
            const uint32_t en = S.ent[k][e];
            const int x = G.ssp[en & 0xff], sh = (en >> 8) & 1;
            const int t = S.eps_q[sh][A * 5 + x] - S.eps_q[sh][kVac * 5 + x];
            atomicAdd(&G.acc32[k], (en >> 9) & 1 ? -t : t);
        }
    } else if (MODE == 1) {
        constexpr int WPH = NW >= 16 ? 2 : 1;
        for (int kk = warp; kk < n * 8 * WPH; kk += NW) {
            const int g = kk / (8 * WPH), r = kk - g * 8 * WPH, k = r & 7, half = r >> 3;
            Grp& G = D.grp[g];
            const int A = G.ssp[S.mk[k]];
            if (A == kVac) continue;
            long long v = 0;
            int bad = 0;
            for (int e = half * 32 + lane; e < kEamE; e += 32 * WPH) {
                const uint32_t en = S.ent[k][e];
                if (en >> 14) {
                    const int mk = S.mk[k];
                    v += embed_q(S, A, G.srho[0] - S.fq[A][1], bad) - G.fsite[mk];
                    bad |= G.fbad[mk];
                } else {
                    const int idx = en & 0xff, sip = (en >> 8) & 7, sim = (en >> 11) & 7;
                    const int a = G.ssp[idx];
                    if (a == kVac) continue;
                    const int pi = pair_index(A, a);
                    v += embed_q(S, a, G.srho[idx] + S.fq[A][sip] - S.fq[A][sim], bad) - G.fsite[idx] +
                         (S.phi_q[pi][sip] - S.phi_q[pi][sim]);
                    bad |= G.fbad[idx];
                }
            }
            v = warp_sum(v);
            bad = __any_sync(0xffffffffu, bad);
            if (lane == 0) {
                G.acc64[half][k] = v;
                if (bad) G.hop_bad[k] = 1;
            }
        }
    } else {
        for (int kk = warp; kk < n * 8; kk += NW) {
            const int g = kk >> 3, k = kk & 7;
            Grp& G = D.grp[g];
            const int A = G.ssp[S.mk[k]];
            if (A == kVac) {
                if (lane == 0) G.hop_de[k] = 0.0;
                continue;
            }
            double acc = 0.0;
            int bad = 0;
            for (int j = lane; j < kEamE; j += 32) {
                const uint32_t en = S.ent[k][j];
                int a, r0, r1;
                double ph = 0.0;
                if (en >> 14) {
                    a = A;
                    r0 = G.srho[S.mk[k]];
                    r1 = G.srho[0] - S.fq[A][1];
                } else {
                    const int idx = en & 0xff, sip = (en >> 8) & 7, sim = (en >> 11) & 7;
                    a = G.ssp[idx];
                    if (a == kVac) continue;
                    r0 = G.srho[idx];
                    r1 = r0 + S.fq[A][sip] - S.fq[A][sim];
                    const int pi = pair_index(A, a);
                    ph = S.phi_d[pi][sip] - S.phi_d[pi][sim];
                }
                acc += (embed_fp64(S, a, r1, bad) - embed_fp64(S, a, r0, bad)) + ph;
            }
            acc = warp_sum(acc);
            bad = __any_sync(0xffffffffu, bad);
            if (lane == 0) {
                G.hop_de[k] = acc;
                G.hop_bad[k] = bad;
            }
        }
    }
}

// R for up to kG vacancies at once: lane 8g + k takes hop k of vacancy g (the
// arithmetic of phase_rates), then lane 0 updates the tree paths one after the
// other.  Only warp 0 executes this; it ends with __syncwarp.
template <int MODE>
__device__ __forceinline__ void grp_rates(StepShared& S, const Dyn& D, int g0, int n) {
    const int lane = threadIdx.x & 31, g = lane >> 3, k = lane & 7;
    const bool on = g < n;
    const int q = on ? grp_vacancy(S, D, g0 + g) : 0;
    const Grp& G = D.grp[on ? g : 0];
    const int A = G.ssp[S.mk[k]];
    double de, gr;
    if (MODE == 2) {
        de = G.hop_de[k];
        gr = hop_rate_fp64(S, D, A, de);
    } else {
        const int dq = MODE == 0 ? G.acc32[k] : (int)((G.acc64[0][k] + G.acc64[1][k] + (1LL << 15)) >> 16);
        de = A == kVac ? 0.0 : (double)dq * 0x1p-24;
        gr = hop_rate_grid(S, D, A, dq);
    }
    const int bad = on && (G.hop_bad[k] | !finite_bits(gr));
    const double s1 = gr + __shfl_xor_sync(0xffffffffu, gr, 1);
    const double s2 = s1 + __shfl_xor_sync(0xffffffffu, s1, 2);
    const double s3 = s2 + __shfl_xor_sync(0xffffffffu, s2, 4);
    const bool anybad = __any_sync(0xffffffffu, bad);
    if (on) {
        D.rates[8 * q + k] = gr;
        D.dE[8 * q + k] = de;
        D.hop_sp[8 * q + k] = (uint8_t)A;
        double* h = D.hsum + 8 * q;
        if ((k & 1) == 0) h[4 + (k >> 1)] = s1;
        if ((k & 3) == 0) h[2 + (k >> 2)] = s2;
        if (k == 0) {
            h[1] = s3;
            D.tree[S.v.P + q] = s3;
        }
    }
    __syncwarp();
    if (lane == 0) {
        const int P = S.v.P;
        for (int gg = 0; gg < n; ++gg) {
            const int qq = grp_vacancy(S, D, g0 + gg);
            for (int i = (P + qq) >> 1; i >= 1; i >>= 1) D.tree[i] = D.tree[2 * i] + D.tree[2 * i + 1];
        }
        if (anybad) S.numeric = 1;
    }
    __syncwarp();
}

// Full refresh of one vacancy with barriers (rebuild, and vacancies other
// than the moved one).
template <int NW, int MODE>
__device__ void refresh_full(StepShared& S, const Dyn& D, int q) {
    phase_gather<NW, MODE>(S, D, q, false);
    __syncthreads();
    if (MODE == 1) {
        phase_site_embed<NW>(S);
        __syncthreads();
    }
    phase_terms<NW, MODE>(S, false);
    __syncthreads();
    if (threadIdx.x < 32) phase_rates<MODE>(S, D, q);
    __syncthreads();
}

// (a9) dt = -ln(u2)/R of the batched events, evaluated lane-parallel, summed
// pairwise (relative error below 10 ulp of the batch sum), and folded into
// the Neumaier-compensated clock (t_hi, t_lo).
template <int NW>
__device__ void flush_clock(StepShared& S) {
    const int tid = threadIdx.x;
    const int cnt = S.ccount;
    if (cnt == 0) return;   // uniform
    for (int i = tid; i < cnt; i += NW * 32) S.cu2[i] = -log(S.cu2[i]) / S.cR[i];
    __syncthreads();
    if (tid < 32) {
        double s = 0.0;
        for (int i = tid; i < cnt; i += 32) s += S.cu2[i];
        s = warp_sum(s);
        if (tid == 0) {
            const double hi = S.t_hi + s;
            if (fabs(S.t_hi) >= fabs(s))
                S.t_lo += (S.t_hi - hi) + s;
            else
                S.t_lo += (s - hi) + S.t_hi;
            S.t_hi = hi;
            S.ccount = 0;
        }
    }
    __syncthreads();
}

template <int NW>
__device__ void load_voxel_state(StepShared& S, const Dyn& D) {
    const int tid = threadIdx.x;
    const VoxelDev& V = S.v;
    const int L = V.L;
    for (int i = tid; i < V.nv; i += NW * 32) {
        int s = V.vac_pos[i];
        int b = s & 1, c = s >> 1;
        D.pos[i] = s;
        D.X[i] = 2 * (c % L) + b;
        D.Y[i] = 2 * ((c / L) % L) + b;
        D.Z[i] = 2 * (c / (L * L)) + b;
    }
    for (int i = tid; i < 3 * V.nv; i += NW * 32) D.disp[i] = V.vac_disp[i];
    for (int i = tid; i < 8 * V.nv; i += NW * 32) {
        D.rates[i] = V.rates[i];
        D.dE[i] = V.dE[i];
        D.hop_sp[i] = V.hop_sp[i];
    }
    for (int i = tid; i < 2 * V.P; i += NW * 32) D.tree[i] = V.tree[i];
    for (int i = tid; i < kEtab; i += NW * 32) D.etab[i] = V.etab[i];
    for (int q = tid; q < V.nv; q += NW * 32) {
        const double* g = V.rates + 8 * q;
        double* h = D.hsum + 8 * q;
        h[4] = g[0] + g[1];
        h[5] = g[2] + g[3];
        h[6] = g[4] + g[5];
        h[7] = g[6] + g[7];
        h[2] = h[4] + h[5];
        h[3] = h[6] + h[7];
        h[1] = h[2] + h[3];
    }
    if (tid == 0) {
        S.t_hi = V.t_hi;
        S.t_lo = V.t_lo;
        S.n = V.n_events;
        S.stop = 0;
        S.numeric = 0;
        S.ccount = 0;
    }
    __syncthreads();
    if (tid == 0) next_uniforms(S);
}

template <int NW>
__device__ void store_voxel_state(StepShared& S, const Dyn& D, VoxelDev* gv) {
    const int tid = threadIdx.x;
    const VoxelDev& V = S.v;
    for (int i = tid; i < V.nv; i += NW * 32) V.vac_pos[i] = D.pos[i];
    for (int i = tid; i < 3 * V.nv; i += NW * 32) V.vac_disp[i] = D.disp[i];
    for (int i = tid; i < 8 * V.nv; i += NW * 32) {
        V.rates[i] = D.rates[i];
        V.dE[i] = D.dE[i];
        V.hop_sp[i] = D.hop_sp[i];
    }
    for (int i = tid; i < 2 * V.P; i += NW * 32) V.tree[i] = D.tree[i];
    if (tid == 0) {
        gv->t_hi = S.t_hi;
        gv->t_lo = S.t_lo;
        gv->n_events = S.n;
        gv->status = S.v.status;
    }
}

// (a6) select with u1 * R (descent compares as integers) and (a7) apply the
// swap; executed by lane 0 of warp 0.  Returns false if the voxel is trapped
// or a numeric error was flagged.
__device__ __forceinline__ bool select_and_swap(StepShared& S, const Dyn& D) {
    const double R = D.tree[1];
    if (S.numeric) {
        S.v.status = kENUMERIC;
        return false;
    }
    if (!(__double_as_longlong(R) > 0)) {
        S.v.status = kETRAPPED;
        return false;
    }
    double t = S.nu1 * R;
    const int P = S.v.P;
    int node = 1;
    while (node < P) {
        const double l = D.tree[2 * node], r = D.tree[2 * node + 1];
        if (lt_nonneg(t, l) || is_zero(r)) {
            node = 2 * node;
        } else {
            t -= l;
            node = 2 * node + 1;
        }
    }
    const int slot = node - P;
    const double* hp = D.hsum + 8 * slot;
    const double* gp = D.rates + 8 * slot;
    const double h2 = hp[2], h3 = hp[3], h4 = hp[4], h5 = hp[5], h6 = hp[6], h7 = hp[7];
    const double g0 = gp[0], g1 = gp[1], g2 = gp[2], g3 = gp[3], g4 = gp[4], g5 = gp[5], g6 = gp[6], g7 = gp[7];
    const unsigned long long hops = *(const unsigned long long*)(D.hop_sp + 8 * slot);
    const int wX = D.X[slot], wY = D.Y[slot], wZ = D.Z[slot], w = D.pos[slot];
    int d = 0;
    if (!(lt_nonneg(t, h2) || is_zero(h3))) { t -= h2; d = 4; }
    const double l2 = d ? h6 : h4, r2 = d ? h7 : h5;
    if (!(lt_nonneg(t, l2) || is_zero(r2))) { t -= l2; d += 2; }
    const double l3 = d == 0 ? g0 : d == 2 ? g2 : d == 4 ? g4 : g6;
    const double r3 = d == 0 ? g1 : d == 2 ? g3 : d == 4 ? g5 : g7;
    if (!(lt_nonneg(t, l3) || is_zero(r3))) d += 1;
    const int L = S.v.L, M2 = 2 * L;
    const int dx = (d & 1) ? -1 : 1, dy = (d & 2) ? -1 : 1, dz = (d & 4) ? -1 : 1;
    const int mX = wrap_coord(wX + dx, M2), mY = wrap_coord(wY + dy, M2), mZ = wrap_coord(wZ + dz, M2);
    const int m = site_index(mX, mY, mZ, L);
    const int A = (int)((hops >> (8 * d)) & 0xff);
    S.v.species[w] = (uint8_t)A;
    S.v.species[m] = (uint8_t)kVac;
    S.slot = slot;
    S.dir = d;
    S.A = A;
    S.wX = wX; S.wY = wY; S.wZ = wZ;
    S.mX = mX; S.mY = mY; S.mZ = mZ;
    S.n_aff = 0;
    D.pos[slot] = m;
    D.X[slot] = mX;
    D.Y[slot] = mY;
    D.Z[slot] = mZ;
    D.disp[3 * slot + 0] += dx;
    D.disp[3 * slot + 1] += dy;
    D.disp[3 * slot + 2] += dz;
    const int c = S.ccount;
    S.cu2[c] = S.nu2;
    S.cR[c] = R;
    S.ccount = c + 1;
    if (S.v.log_cap > 0) S.v.log[S.n % (uint64_t)S.v.log_cap] = 8 * slot + d;
    S.n += 1;
    return true;
}

// Events of the resident voxel (a6 -> a7 -> a8, a9 batched), target at most.
// Per event: [warp 0: select + swap] B [gather, affected list, next Philox]
// B ([site embedding] B) [hop terms, density updates] B [warp 0: rates + tree];
// warp 0 goes straight on to the next select, so the rates of event n and the
// selection of event n+1 need no CTA-wide barrier between them.
template <int NW, int MODE>
__device__ void run_events(StepShared& S, const Dyn& D, uint64_t target) {
    const int tid = threadIdx.x;
    const int L = S.v.L;
    int ccount = S.ccount;   // uniform copy of the clock-batch fill
    const bool fast = S.v.nv == 1 && L >= (MODE != 0 ? 6 : 5);
    if (fast) {
        phase_prefetch<NW, MODE>(S, D, 0);
        __syncthreads();
    }
    for (uint64_t done = 0; done < target; ++done) {
        if (tid == 0) S.stop = !select_and_swap(S, D);
        __syncthreads();
        if (S.stop) break;
        ++ccount;
        if (fast) {
            phase_fill<NW, MODE>(S);
            __syncthreads();
            phase_terms<NW, MODE>(S, true);
            __syncthreads();
            if (tid < 32) phase_rates<MODE>(S, D, S.slot);
            phase_prefetch<NW, MODE>(S, D, NW > 1 ? 32 : 0);
        } else {
            // (a7) the hop's density updates and (a8) the refresh list, then the
            // moved vacancy and every vacancy within reach, kG per pass
            phase_hop_update<NW, MODE>(S, D);
            __syncthreads();
            const int n_all = 1 + S.n_aff;
            for (int g0 = 0; g0 < n_all; g0 += kG) {
                const int n = min(kG, n_all - g0);
                grp_gather<NW, MODE>(S, D, g0, n);
                __syncthreads();
                if (MODE == 1) {
                    grp_site_embed<NW>(S, D, n);
                    __syncthreads();
                }
                grp_terms<NW, MODE>(S, D, n);
                __syncthreads();
                if (tid < 32) grp_rates<MODE>(S, D, g0, n);
                if (g0 + kG < n_all) __syncthreads();
            }
        }
        if (ccount == kClockBatch) {
            flush_clock<NW>(S);
            ccount = 0;
        }
    }
    __syncthreads();
    if (tid == 0 && S.numeric && S.v.status == kOK) S.v.status = kENUMERIC;
    flush_clock<NW>(S);
}

// ---- single-vacancy path: lattice window in shared memory -------------------
// A voxel with one vacancy keeps a window of W^3 cells (W = min(L, 16); species
// and, for EAM, densities) around the vacancy in shared memory, so no read of
// an event touches global memory.  Every change is written through to the
// lattice in global memory as well (species stores, density atomics), and the
// window is reloaded, centred on the vacancy, when the vacancy comes within 2
// cells of its edge (all stencils of the vacancy and of its 8 targets reach at
// most 4 half units).  An event takes two phases:
//  A  warp 0: the 8 rates from the hop sums (a4), their subtree sums (a5) and
//     the selection (a6) in lanes 0..7, then the swap (a7); the vacancy's
//     coordinates live in registers and the 8 candidate moves are prepared
//     lane-parallel while the float64 chain runs (on GB300 every float64 warp
//     instruction holds the SM sub-partition's FP64 pipe for ~64 cycles, so
//     the chain is kept to the operations the rate arithmetic needs);
//     meanwhile the other warps add the previous hop's density change (a7) to
//     the window and to memory and draw the uniforms of the next event;
//  B  every warp: the energy changes of the 8 hops of the moved vacancy (a2,
//     a3), reading the window (which lags by the hop just made) and adding
//     that hop's density change from a table; one warp (two for 16 warps) per
//     hop, exact integer sums reduced with warp reductions.
// The arithmetic of every rate, sum and comparison is the one of the general
// path, so the two give identical trajectories.

// Window layout: a row (fixed cell y, z) holds the 2W sites X = 2x + b in order;
// rows are padded to 2W + 1 sites and planes to W (2W + 1) + 8, so that sites
// in neighbouring rows and planes fall in different shared-memory banks.
__host__ __device__ inline int win_sites(int W) { return W * (W * (2 * W + 1) + 8); }

__device__ __forceinline__ int widx(int X, int Y, int Z, int W) {
    const int RS = 2 * W + 1, PS = W * RS + 8;
    return (Z >> 1) * PS + (Y >> 1) * RS + X;
}

// Window-index difference of the site at packed offset o from a site of parity b.
__device__ __forceinline__ int wdelta(int b, int32_t o, int W) {
    const int B = 4 + b;
    return widx(B + off_dx(o), B + off_dy(o), B + off_dz(o), W) - widx(B, B, B, W);
}

// Thread 0: centre the window on the vacancy at global half-unit (X, Y, Z).
__device__ __forceinline__ void window_center(StepShared& S, int X, int Y, int Z) {
    const int W = S.W, L = S.v.L;
    auto org = [&](int G) { const int o = (G >> 1) - W / 2; return o < 0 ? o + L : o; };
    auto loc = [&](int G, int o) { const int l = G - 2 * o; return l < 0 ? l + 2 * L : l; };
    S.ox = org(X);
    S.oy = org(Y);
    S.oz = org(Z);
    S.lX = loc(X, S.ox);
    S.lY = loc(Y, S.oy);
    S.lZ = loc(Z, S.oz);
    S.wb = widx(S.lX, S.lY, S.lZ, W);
}

// All threads: load the window at the current origin (L2 loads that bypass L1,
// so the density atomics of this CTA are seen).  One warp per window row
// (cells y, z; its 2W sites are contiguous in the lattice unless x wraps), the
// lanes over the row's sites, four rows in flight per warp.
template <int NW, int MODE>
__device__ void window_load(StepShared& S, const Dyn& D) {
    const int W = S.W, L = S.v.L, ox = S.ox, oy = S.oy, oz = S.oz;
    const int M2 = 2 * L, W2 = 2 * W, RS = 2 * W + 1, PS = W * RS + 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint8_t* sp = S.v.species;
    const int32_t* rho = S.v.rho;
    // this lane's site of a row: cell lx = c / 2, parity c & 1, lattice x wrapped once
    const int c = lane;
    int gx = ox + (c >> 1);
    gx -= gx >= L ? L : 0;
    const int xoff = 2 * gx + (c & 1);
    const bool on = c < W2;
    const int n_rows = W * W;
    for (int r0 = warp; r0 < n_rows; r0 += 4 * NW) {
        uint8_t s4[4];
        int32_t q4[4];
        int w4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + u * NW;
            const bool ok = on && r < n_rows;
            const int ly = r % W, lz = r / W;
            int gy = oy + ly, gz = oz + lz;
            gy -= gy >= L ? L : 0;
            gz -= gz >= L ? L : 0;
            const size_t g = ((size_t)gz * L + gy) * M2 + xoff;
            w4[u] = ok ? lz * PS + ly * RS + c : -1;
            s4[u] = ok ? __ldcg(sp + g) : 0;
            if (MODE != 0) q4[u] = ok ? __ldcg(rho + g) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (w4[u] >= 0) {
                D.wsp[w4[u]] = s4[u];
                if (MODE != 0) D.wrho[w4[u]] = q4[u];
            }
    }
}

// Exact sum over the warp of integers below 2^48 in magnitude (two 32-bit
// warp reductions: of the low 24 bits and of the rest).
__device__ __forceinline__ long long warp_sum_exact(long long v) {
    const unsigned lo = (unsigned)(v & 0xFFFFFF);
    const int hi = (int)(v >> 24);
    const unsigned slo = __reduce_add_sync(0xffffffffu, lo);
    const int shi = __reduce_add_sync(0xffffffffu, hi);
    return (long long)shi * 16777216LL + (long long)slo;
}

// The float64 value q * 2^-24 of an integer q, built from its bits (exact).
__device__ __forceinline__ double q24_to_double(int q) {
    if (q == 0) return 0.0;
    const unsigned long long m = q < 0 ? (unsigned long long)(-(long long)q) : (unsigned long long)q;
    const int e = 63 - __clzll((long long)m);                 // top bit, < 32
    const unsigned long long mant = (m << (52 - e)) & 0xFFFFFFFFFFFFFull;
    const unsigned long long bits = ((unsigned long long)(e - 24 + 1023) << 52) | mant |
                                    (q < 0 ? 0x8000000000000000ull : 0ull);
    return __longlong_as_double((long long)bits);
}

template <int NW, int MODE>
__device__ void run_events_window(StepShared& S, const Dyn& D, uint64_t target) {
    static_assert(NW == 8 || NW == 16, "window path: 8 or 16 warps");
    static_assert(MODE == 0 || MODE == 1, "window path: pair model or split-precision EAM");
    constexpr int NT = NW * 32;
    constexpr int WPH = NW / 8;                                     // warps per hop
    constexpr int NE = MODE == 0 ? kPairE : kEamE;                  // entries per hop
    constexpr int EJ = (NE + 32 * WPH - 1) / (32 * WPH);            // entries per lane
    // roles by rotated thread index: a second CTA on the SM puts its warp 0
    // (the float64 chain of phase A) on another sub-partition (see sm_rotation)
    const int tid = (threadIdx.x + S.wrot) & (NT - 1), lane = tid & 31, warp = tid >> 5;
    const int L = S.v.L, M2 = 2 * L;
    if (tid == 0) {
        S.W = L < kWinMax ? L : kWinMax;
        window_center(S, D.X[0], D.Y[0], D.Z[0]);
    }
    // density change of a hop in direction d of atom A at read-set site u:
    // dprev[(d * 4 + A) * kEamU + u] = f_A(r_uw) - f_A(r_um) (u fastest, so the
    // lanes of a warp, which read different sites, hit different banks)
    if (MODE != 0)
        for (int i = tid; i < kEamU * 32; i += NT) {
            const int u = i % kEamU, da = i / kEamU, d = da >> 2, A = da & 3;
            const int ds = S.dsh[u][d];
            D.dprev[i] = S.fq[A][ds >> 3] - S.fq[A][ds & 7];
        }
    __syncthreads();
    const int W = S.W;
    window_load<NW, MODE>(S, D);
    // per-lane constants of phase B: entries of hop k = warp % 8 and their
    // window offsets for both parities of the vacancy site
    const int k = warp & 7, half = warp >> 3;
    uint32_t en[EJ];
    int dl0[EJ], dl1[EJ];
#pragma unroll
    for (int j = 0; j < EJ; ++j) {
        const int e = half * 32 + lane + 32 * WPH * j;
        en[j] = e < NE ? S.ent[k][e] : 0xFFFFFFFFu;
        const bool site = e < NE && (MODE == 0 || !(en[j] >> 14));
        const int32_t o = site ? S.off[en[j] & 0xff] : off_pack(0, 0, 0, 0);
        dl0[j] = wdelta(0, o, W);
        dl1[j] = wdelta(1, o, W);
    }
    // the lane holding the hop's own-embedding entry (one per hop)
    bool own_lane = false;
#pragma unroll
    for (int j = 0; j < EJ; ++j) own_lane |= MODE != 0 && en[j] != 0xFFFFFFFFu && (en[j] >> 14);
    const int32_t omk = S.off[S.mk[k]];
    const int dm0 = wdelta(0, omk, W), dm1 = wdelta(1, omk, W);
    // embedding of the read set's sites (split-precision EAM): thread u takes
    // union site u around the vacancy
    const bool sf_on = MODE != 0 && tid < kEamU;
    const int32_t sfo = sf_on ? S.off[tid] : off_pack(0, 0, 0, 0);
    const int sf0 = wdelta(0, sfo, W), sf1 = wdelta(1, sfo, W);
    const int mkk = S.mk[k];
    const EmbedC E = embed_consts(S);
    // per-thread constants of the density update: threads of the warps that do
    // not share warp 0's SM sub-partition (warp % 4 != 0), in order
    const int ut = (warp & 3) ? (warp - 1 - warp / 4) * 32 + lane : -1;
    const bool upd = MODE != 0 && ut >= 0 && ut < 2 * kSph;
    const int uside = upd && ut >= kSph;
    const int32_t uo = upd ? S.sph[uside ? ut - kSph : ut] : off_pack(0, 0, 0, 0);
    const int ud0 = wdelta(0, uo, W), ud1 = wdelta(1, uo, W), ush = off_extra(uo);
    // warp 0: the vacancy in registers; lane k's candidate move d = k
    const int cdx = (lane & 1) ? -1 : 1, cdy = (lane & 2) ? -1 : 1, cdz = (lane & 4) ? -1 : 1;
    int gX = D.X[0], gY = D.Y[0], gZ = D.Z[0], lX = S.lX, lY = S.lY, lZ = S.lZ, wb = S.wb, pos = D.pos[0];
    int disp0 = D.disp[0], disp1 = D.disp[1], disp2 = D.disp[2];
    uint64_t n_ev = S.n;
    const int log_cap = S.v.log_cap;
    int32_t* const log = S.v.log;
    uint8_t* const species = S.v.species;
    const int hi_edge = 2 * W - 5;
    const bool etab_ok = S.v.etab_ok;
    __syncthreads();

    int ccount = S.ccount;
    uint64_t n_next = S.n + 1;       // event index whose uniforms the next phase A draws
    bool first = true;
    for (uint64_t done = 0;; ++done) {
        const bool finish = done >= target;
        // ---------------- phase A
        if (warp == 0) {
            if (lane < 8) {
                // candidate move of this lane (integer work beside the float64 chain)
                const int mX = wrap_coord(gX + cdx, M2), mY = wrap_coord(gY + cdy, M2), mZ = wrap_coord(gZ + cdz, M2);
                const int mpos = site_index(mX, mY, mZ, L);
                const int mlX = lX + cdx, mlY = lY + cdy, mlZ = lZ + cdz;
                const int mwb = widx(mlX, mlY, mlZ, W);
                const bool out = mlX < 4 || mlX > hi_edge || mlY < 4 || mlY > hi_edge || mlZ < 4 || mlZ > hi_edge;
                const double u1 = S.nu1, u2 = S.nu2;
                int A, dq = 0, bad, d = 0;
                bool trapped;
                double g = 0.0, R = 0.0;
                if constexpr (WPH == 1) {
                    // (a4)+(a6) in integers: the float64 rates, their sum for the clock
                    // and the stored state come from warp 4 beside this chain
                    unsigned long long M;
                    int E;
                    if (first) {
                        A = D.hop_sp[lane];
                        g = D.rates[lane];
                        bad = !finite_bits(g);
                        rate_to_fixed(g, M, E);
                    } else {
                        A = S.hsp[lane];
                        dq = MODE == 0 ? S.acc32[lane] : (int)((S.acc64[0][lane] + S.acc64[1][lane] + (1LL << 15)) >> 16);
                        bad = S.hbad[0][lane] | S.hbad[1][lane];
                        hop_rate_fixed(S, D, A, dq, etab_ok, M, E, bad);
                    }
                    bad = __any_sync(0xffu, bad);
                    // every rate on the scale of the largest (below 2^60, the others
                    // truncated below 2^-60 of it), inclusive prefix sums over the lanes,
                    // t = floor(u1 R), and the first lane whose prefix exceeds t: the
                    // event the float64 tree descent picks unless t lies within rounding
                    // of a boundary (a declared tie)
                    const int Em = __reduce_max_sync(0xffu, M ? E : -(1 << 20));
                    const int sh = Em - E + 4;
                    unsigned long long P = (M == 0 || sh >= 64) ? 0ull : M >> sh;
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1) {
                        const unsigned long long x = __shfl_up_sync(0xffu, P, o);
                        if (lane >= o) P += x;
                    }
                    const unsigned long long Rq = __shfl_sync(0xffu, P, 7);
                    const unsigned long long tq = __umul64hi(S.nuU1 << 11, Rq);
                    d = __ffs(__ballot_sync(0xffu, tq < P)) - 1;
                    trapped = Rq == 0;
                } else {
                    if (first) {
                        A = D.hop_sp[lane];
                        g = D.rates[lane];
                        bad = !finite_bits(g);
                    } else {
                        A = S.hsp[lane];
                        dq = MODE == 0 ? S.acc32[lane] : (int)((S.acc64[0][lane] + S.acc64[1][lane] + (1LL << 15)) >> 16);
                        g = hop_rate_grid(S, D, A, dq);
                        bad = S.hbad[0][lane] | S.hbad[1][lane] | !finite_bits(g);
                    }
                    const double s1 = g + __shfl_xor_sync(0xffu, g, 1);
                    const double s2 = s1 + __shfl_xor_sync(0xffu, s1, 2);
                    R = s2 + __shfl_xor_sync(0xffu, s2, 4);
                    bad = __any_sync(0xffu, bad);
                    // (a6) descent over the 3 levels of the vacancy's hop tree, the
                    // compares and subtractions of the general path, in every lane
                    double t = u1 * R;
                    const double h2 = __shfl_sync(0xffu, s2, 0), h3 = __shfl_sync(0xffu, s2, 4);
                    const double h4 = __shfl_sync(0xffu, s1, 0), h5 = __shfl_sync(0xffu, s1, 2);
                    const double h6 = __shfl_sync(0xffu, s1, 4), h7 = __shfl_sync(0xffu, s1, 6);
                    const double g0 = __shfl_sync(0xffu, g, 0), g1 = __shfl_sync(0xffu, g, 1);
                    const double g2 = __shfl_sync(0xffu, g, 2), g3 = __shfl_sync(0xffu, g, 3);
                    const double g4 = __shfl_sync(0xffu, g, 4), g5 = __shfl_sync(0xffu, g, 5);
                    const double g6 = __shfl_sync(0xffu, g, 6), g7 = __shfl_sync(0xffu, g, 7);
                    if (!(lt_nonneg(t, h2) || is_zero(h3))) { t -= h2; d = 4; }
                    const double l2 = d ? h6 : h4, r2 = d ? h7 : h5;
                    if (!(lt_nonneg(t, l2) || is_zero(r2))) { t -= l2; d += 2; }
                    const double l3 = d == 0 ? g0 : d == 2 ? g2 : d == 4 ? g4 : g6;
                    const double r3 = d == 0 ? g1 : d == 2 ? g3 : d == 4 ? g5 : g7;
                    if (!(lt_nonneg(t, l3) || is_zero(r3))) d += 1;
                    trapped = !(__double_as_longlong(R) > 0);
                    // stored state of this event's rates (off the chain)
                    D.rates[lane] = g;
                    D.dE[lane] = (A == kVac || first) ? (first ? D.dE[lane] : 0.0) : q24_to_double(dq);
                    D.hop_sp[lane] = (uint8_t)A;
                }
                const bool go = !finish && !bad && !S.numeric && !trapped;
                if (go) {
                    // (a7) the move of lane d: vacancy w -> m, atom Ad m -> w
                    const int Ad = __shfl_sync(0xffu, A, d);
                    const int nX = __shfl_sync(0xffu, mX, d), nY = __shfl_sync(0xffu, mY, d);
                    const int nZ = __shfl_sync(0xffu, mZ, d), npos = __shfl_sync(0xffu, mpos, d);
                    const int nlX = __shfl_sync(0xffu, mlX, d), nlY = __shfl_sync(0xffu, mlY, d);
                    const int nlZ = __shfl_sync(0xffu, mlZ, d), nwb = __shfl_sync(0xffu, mwb, d);
                    const bool nout = __shfl_sync(0xffu, out, d);
                    if (lane == 0) {
                        D.wsp[wb] = (uint8_t)Ad;
                        D.wsp[nwb] = (uint8_t)kVac;
                        species[pos] = (uint8_t)Ad;
                        species[npos] = (uint8_t)kVac;
                        S.dir = d;
                        S.A = Ad;
                        S.wX = gX; S.wY = gY; S.wZ = gZ;
                        S.mX = nX; S.mY = nY; S.mZ = nZ;
                        S.lX = nlX; S.lY = nlY; S.lZ = nlZ;
                        S.wb = nwb;
                        S.recenter = nout;
                        const int c = ccount;
                        S.cu2[c] = u2;
                        if constexpr (WPH != 1) S.cR[c] = R;
                        if (log_cap > 0) log[n_ev % (uint64_t)log_cap] = d;
                    }
                    disp0 += (d & 1) ? -1 : 1;
                    disp1 += (d & 2) ? -1 : 1;
                    disp2 += (d & 4) ? -1 : 1;
                    gX = nX; gY = nY; gZ = nZ;
                    lX = nlX; lY = nlY; lZ = nlZ;
                    wb = nwb;
                    pos = npos;
                    n_ev += 1;
                }
                if (lane == 0) {
                    if constexpr (WPH != 1) D.tree[1] = R;
                    if (bad) S.numeric = 1;
                    if (!finish && !go) {
                        S.v.status = (bad || S.numeric) ? kENUMERIC : kETRAPPED;
                        S.stop = 1;
                    }
                    if (finish || !go) {
                        S.recenter = 0;
                        S.n = n_ev;
                        S.ccount = ccount;
                        D.pos[0] = pos;
                        D.X[0] = gX;
                        D.Y[0] = gY;
                        D.Z[0] = gZ;
                        D.disp[0] = disp0;
                        D.disp[1] = disp1;
                        D.disp[2] = disp2;
                    }
                }
            }
        } else {
            if constexpr (WPH == 1) {
                if (warp == 4 && lane < 8) {
                    // the float64 rates of this event (stored state), their sum for
                    // the clock and the stored tree root, as the general path computes them
                    double g;
                    if (first) {
                        g = D.rates[lane];
                    } else {
                        const int A = S.hsp[lane];
                        const int dq = MODE == 0 ? S.acc32[lane]
                                                 : (int)((S.acc64[0][lane] + S.acc64[1][lane] + (1LL << 15)) >> 16);
                        g = hop_rate_grid(S, D, A, dq);
                        D.rates[lane] = g;
                        D.dE[lane] = A == kVac ? 0.0 : q24_to_double(dq);
                        D.hop_sp[lane] = (uint8_t)A;
                    }
                    const double s1 = g + __shfl_xor_sync(0xffu, g, 1);
                    const double s2 = s1 + __shfl_xor_sync(0xffu, s1, 2);
                    const double R = s2 + __shfl_xor_sync(0xffu, s2, 4);
                    if (lane == 0) {
                        S.cR[ccount] = R;
                        D.tree[1] = R;
                    }
                }
            }
            if (upd && !first) {
                // (a7) density change of the pending hop w -> m (atom pA now at w):
                // rho_i += f_A(r_iw) over S(w), -= f_A(r_im) over S(m)
                const int c = uside ? S.pm : S.pw, cb = uside ? S.pmb : S.pwb;
                const int f = S.fq[S.pA][ush];
                atomicAdd(&D.wrho[c + (cb ? ud1 : ud0)], uside ? -f : f);
                const int cX = uside ? S.pmX : S.pwX, cY = uside ? S.pmY : S.pwY, cZ = uside ? S.pmZ : S.pwZ;
                const int s = site_index(wrap_coord(cX + off_dx(uo), M2), wrap_coord(cY + off_dy(uo), M2),
                                         wrap_coord(cZ + off_dz(uo), M2), L);
                atomicAdd(&S.v.rho[s], uside ? -f : f);
            }
            if (tid == NT - 1 && !finish) {
                // uniforms of the event after the one selected in this phase
                const uint64_t uid = S.v.uid, seed = S.v.seed;
                uint32_t c0 = (uint32_t)n_next, c1 = (uint32_t)(n_next >> 32), c2 = (uint32_t)uid,
                         c3 = (uint32_t)(uid >> 32) & 0x7fffffffu;
                philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
                S.nxU1 = ((uint64_t)c0 << 21) | (c1 >> 11);
                S.nx1 = u53_to_double(S.nxU1);
                S.nx2 = u53_to_double((((uint64_t)c2 << 21) | (c3 >> 11)) + 1);
            }
        }
        __syncthreads();
        if (finish || S.stop) break;
        first = false;
        ++ccount;
        ++n_next;
        if (S.recenter) {
            if (tid == 0) window_center(S, S.mX, S.mY, S.mZ);
            __syncthreads();
            window_load<NW, MODE>(S, D);
            if (warp == 0) {
                lX = S.lX;
                lY = S.lY;
                lZ = S.lZ;
                wb = S.wb;
            }
            __syncthreads();
        }
        // ---------------- phase B
        const int b = S.lX & 1, base = S.wb;
        const int Ap = S.A, dp = S.dir;
        const int A = D.wsp[base + (b ? dm1 : dm0)];
        if (MODE != 0) {
            // F_{s_u}(rho_u) of every read-set site at its current density (the
            // window lags by the hop just made; that hop's density change comes from
            // the table), shared by the terms of all 8 hops
            if (sf_on) {
                const int wi = base + (b ? sf1 : sf0);
                const int a = D.wsp[wi];
                int fb = 0;
                const long long f = a != kVac ? embed_c(E, a, D.wrho[wi] + D.dprev[(dp * 4 + Ap) * kEamU + tid], fb) : 0;
                S.fsite[tid] = fb ? kFBad : f;      // a density off the table: flagged in the value
            }
            __syncthreads();
        }
        if (MODE == 0) {
            int v = 0;
            if (A != kVac) {
#pragma unroll
                for (int j = 0; j < EJ; ++j) {
                    const uint32_t e = en[j];
                    if (e == 0xFFFFFFFFu) continue;
                    const int x = D.wsp[base + (b ? dl1[j] : dl0[j])], sh = (e >> 8) & 1;
                    const int t = S.eps_q[sh][A * 5 + x] - S.eps_q[sh][kVac * 5 + x];
                    v += (e >> 9) & 1 ? -t : t;
                }
            }
            v = __reduce_add_sync(0xffffffffu, v);
            if (lane == 0 && half == 0) {
                S.acc32[k] = v;
                S.hsp[k] = A;
                S.hbad[0][k] = S.hbad[1][k] = 0;
            }
        } else {
            long long v = 0;
            int bad = 0;
            if (A != kVac) {
                const int* dpv = D.dprev + (dp * 4 + Ap) * kEamU;
                const int32_t* dkA = S.dkq[A];
                // every load of this lane's entries first (independent chains), then
                // the embedding differences (F at the changed density minus the site's
                // F from the table above) and pair terms of the admissible ones
                int ea[EJ], eu[EJ], es[EJ];
                long long ph[EJ];
                bool on[EJ];
#pragma unroll
                for (int j = 0; j < EJ; ++j) {
                    const uint32_t e = en[j];
                    const bool site = e != 0xFFFFFFFFu && !(e >> 14);
                    const int idx = site ? (int)(e & 0xff) : 0;
                    const int ss = site ? (int)((e >> 8) & 63) : 0;     // sip + 8 sim
                    const int wi = base + (b ? dl1[j] : dl0[j]);
                    const int a = D.wsp[wi];
                    const int r = D.wrho[wi] + dpv[idx];
                    on[j] = site && a != kVac;
                    es[j] = a;
                    eu[j] = idx;
                    ea[j] = r + dkA[ss];
                    ph[j] = S.dphi[pair_index(A, a < kVac ? a : 0)][ss];
                }
#pragma unroll
                for (int j = 0; j < EJ; ++j)
                    if (on[j]) {
                        const long long f = S.fsite[eu[j]];
                        bad |= f == kFBad;
                        v += embed_c(E, es[j], ea[j], bad) - (f == kFBad ? 0 : f) + ph[j];
                    }
                if (own_lane) {
                    // the moving atom's own embedding: F_A(rho_w - f_A(1nn)) - F_A(rho_m)
                    const int rp = D.wrho[base] + dpv[0];
                    const long long f = S.fsite[mkk];
                    bad |= f == kFBad;
                    v += embed_c(E, A, rp - S.fq[A][1], bad) - (f == kFBad ? 0 : f);
                }
            }
            v = warp_sum_exact(v);
            bad = __any_sync(0xffffffffu, bad);
            if (lane == 0) {
                S.acc64[half][k] = v;
                S.hbad[half][k] = bad;
                if (WPH == 1) {
                    S.acc64[1][k] = 0;
                    S.hbad[1][k] = 0;
                }
                if (half == 0) S.hsp[k] = A;
            }
        }
        if (tid == NT - 1) {
            S.nu1 = S.nx1;
            S.nuU1 = S.nxU1;
            S.nu2 = S.nx2;
            // the hop just made becomes the pending density change (window sites
            // taken in the window as it is now, after any re-centring)
            const int d = S.dir;
            const int dx = (d & 1) ? -1 : 1, dy = (d & 2) ? -1 : 1, dz = (d & 4) ? -1 : 1;
            S.pA = S.A;
            S.pm = S.wb;
            S.pmb = S.lX & 1;
            S.pw = widx(S.lX - dx, S.lY - dy, S.lZ - dz, W);
            S.pwb = S.pmb ^ 1;
            S.pwX = S.wX; S.pwY = S.wY; S.pwZ = S.wZ;
            S.pmX = S.mX; S.pmY = S.mY; S.pmZ = S.mZ;
        }
        __syncthreads();
        if (ccount == kClockBatch) {
            if (tid == 0) S.ccount = ccount;
            __syncthreads();
            flush_clock<NW>(S);
            ccount = 0;
        }
    }
    __syncthreads();
    if (tid == 0 && S.numeric && S.v.status == kOK) S.v.status = kENUMERIC;
    flush_clock<NW>(S);
}

// Warps of an SM are spread over its 4 sub-partitions by warp slot; two CTAs
// resident on one SM would put both warps 0, and so both float64 chains of the
// window path, on the same sub-partition and its float64 pipe.  The CTAs that
// arrive on an SM alternate between two rotations of the warp roles (0 and 2
// warps), counted per SM since the library was loaded.
__device__ unsigned int g_sm_arrivals[1024];

__device__ __forceinline__ int sm_rotation() {
    unsigned int sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    return (atomicAdd(&g_sm_arrivals[sm & 1023u], 1u) & 1u) ? 64 : 0;
}

template <int NW>
__global__ void __launch_bounds__(NW * 32) step_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    __shared__ StepShared S;
    const Dyn D = carve(dyn_raw, a.max_nv, a.max_P, a.win);
    load_model<NW>(S, a.model);
    if (threadIdx.x == 0) S.wrot = sm_rotation();
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t h = atomicAdd(a.queue, 1u);
            S.vid = h < (uint32_t)a.n_vox ? a.order[h] : -1;
            if (S.vid >= 0) {
                S.v = a.vox[S.vid];
                S.target = a.targets[S.vid];
            }
        }
        __syncthreads();
        const int vid = S.vid;
        if (vid < 0) break;
        if (S.v.status == kOK && S.target > 0) {
            load_tables<NW>(S, a.tab, S.v.model, S.v.L == 4);
            load_voxel_state<NW>(S, D);
            __syncthreads();
            const int mode = S.v.model == 0 ? 0 : (S.v.precision == 1 ? 1 : 2);
            bool done = false;
            if constexpr (NW >= 8) {
                if (a.win > 0 && window_edge(S.v.L, S.v.nv, S.v.model, S.v.precision) > 0) {
                    if (mode == 0)
                        run_events_window<NW, 0>(S, D, S.target);
                    else
                        run_events_window<NW, 1>(S, D, S.target);
                    done = true;
                }
            }
            if (!done) {
                if (mode == 0)
                    run_events<NW, 0>(S, D, S.target);
                else if (mode == 1)
                    run_events<NW, 1>(S, D, S.target);
                else
                    run_events<NW, 2>(S, D, S.target);
            }
            store_voxel_state<NW>(S, D, &a.vox[vid]);
        }
        __syncthreads();
    }
}

// ---- synchronous sublattice superstep (intra-voxel parallel AKMC) ----------
// The voxel is cut into sectors of Sc^3 cells and each sector into 8 octants of
// (Sc/2)^3 cells.  Superstep k evolves octant k mod 8 (bit 0: upper half in x,
// bit 1: y, bit 2: z) of every sector, one CTA per sector: a local KMC over the
// vacancies inside the octant at the superstep start, with a local clock from
// 0, stopping before the first event whose time would pass the window T; a
// vacancy that leaves the octant drops out (rate 0) for the rest of the
// superstep.  An event reads at most 4 half units beyond its vacancy and
// writes at most 4 half units beyond its start site (hop 1 + cutoff sphere 3),
// while active octants are Sc + 1 half units apart, so for Sc >= 8 the CTAs of
// one superstep touch disjoint sites and need no synchronisation; kernel
// boundaries order the supersteps.  A cycle of 8 supersteps evolves every
// region for T (first-order splitting of the master equation into octant
// parts): the voxel clock advances by T/8 per superstep.

__device__ __forceinline__ bool sl_inside(const StepShared& S, int X, int Y, int Z) {
    const int x = (X >> 1) - S.sl_x0, y = (Y >> 1) - S.sl_y0, z = (Z >> 1) - S.sl_z0, h = S.sl_h;
    return (unsigned)x < (unsigned)h && (unsigned)y < (unsigned)h && (unsigned)z < (unsigned)h;
}

// Time step and window test, then (a6)/(a7) as in the regular path; executed by
// thread 0.  Returns false when no active vacancy has a positive rate, when
// the next event would pass the window, or on a numeric error.
__device__ __forceinline__ bool sl_select(StepShared& S, const Dyn& D) {
    if (S.numeric) {
        S.v.status = kENUMERIC;
        return false;
    }
    const double R = D.tree[1];
    if (!(__double_as_longlong(R) > 0)) return false;
    const double dt = -log(S.nu2) / R;
    const double t = S.sl_t + dt;
    if (t > S.sl_T) return false;
    S.sl_t = t;
    const bool ok = select_and_swap(S, D);
    S.ccount = 0;   // the voxel clock does not take the octant's time steps
    return ok;
}

// Events of one active octant (the loop of run_events with the window test,
// and only the vacancies still inside the octant in the rate tree).
template <int NW, int MODE>
__device__ void run_events_sl(StepShared& S, const Dyn& D) {
    const int tid = threadIdx.x;
    const int L = S.v.L, M2 = 2 * L;
    constexpr int reach = MODE != 0 ? 8 : 4;
    const bool fast = S.v.nv == 1;
    if (fast) {
        phase_prefetch<NW, MODE>(S, D, 0);
        __syncthreads();
    }
    for (;;) {
        if (tid == 0) S.stop = !sl_select(S, D);
        __syncthreads();
        if (S.stop) break;
        // vacancies outside this sector's list whose read set the hop may change
        // (within `reach` half units of w): their stored rates go out of date
        if (tid >= 32) {
            for (int q = tid - 32; q < S.sl_nvtot; q += NW * 32 - 32) {
                if (D.lmap[q] >= 0) continue;
                const int a = D.apos[q];
                int ddx = (a & 1023) - S.wX, ddy = ((a >> 10) & 1023) - S.wY, ddz = (a >> 20) - S.wZ;
                ddx = ddx >= L ? ddx - M2 : (ddx < -L ? ddx + M2 : ddx);
                ddy = ddy >= L ? ddy - M2 : (ddy < -L ? ddy + M2 : ddy);
                ddz = ddz >= L ? ddz - M2 : (ddz < -L ? ddz + M2 : ddz);
                if (abs(ddx) <= reach && abs(ddy) <= reach && abs(ddz) <= reach) S.sl_stale[q] = 1;
            }
        }
        if (fast) {
            phase_fill<NW, MODE>(S);
            __syncthreads();
        } else {
            for (int q = tid; q < S.v.nv; q += NW * 32) {
                if (q == S.slot || !D.on[q]) continue;
                int ddx = D.X[q] - S.wX, ddy = D.Y[q] - S.wY, ddz = D.Z[q] - S.wZ;
                ddx = ddx >= L ? ddx - M2 : (ddx < -L ? ddx + M2 : ddx);
                ddy = ddy >= L ? ddy - M2 : (ddy < -L ? ddy + M2 : ddy);
                ddz = ddz >= L ? ddz - M2 : (ddz < -L ? ddz + M2 : ddz);
                if (abs(ddx) <= reach && abs(ddy) <= reach && abs(ddz) <= reach)
                    D.aff[atomicAdd(&S.n_aff, 1)] = q;
            }
            phase_gather<NW, MODE>(S, D, S.slot, true);
            __syncthreads();
            if (MODE == 1) {
                phase_site_embed<NW>(S);
                __syncthreads();
            }
        }
        phase_terms<NW, MODE>(S, true);
        __syncthreads();
        if (tid < 32) {
            phase_rates<MODE>(S, D, S.slot);
            if (tid == 0) {
                const int q = S.slot;
                if (!sl_inside(S, D.X[q], D.Y[q], D.Z[q])) {
                    D.on[q] = 0;
                    const int P = S.v.P;
                    D.tree[P + q] = 0.0;
                    for (int i = (P + q) >> 1; i >= 1; i >>= 1) D.tree[i] = D.tree[2 * i] + D.tree[2 * i + 1];
                }
            }
        }
        if (fast) phase_prefetch<NW, MODE>(S, D, NW > 1 ? 32 : 0);
        const int n_aff = fast ? 0 : S.n_aff;
        if (n_aff > 0) {
            __syncthreads();
            for (int i = 0; i < n_aff; ++i) refresh_full<NW, MODE>(S, D, D.aff[i]);
        }
    }
    __syncthreads();
}

// One sector's share of superstep k: the vacancies inside its active octant
// (slot order), their rates from the current lattice, then the events.
// Returns the events made (uniform).  Lattice, densities and vacancy records
// are read with L2-only loads (other CTAs write them during the asynchronous
// kernel).  S.v must hold the voxel, S.sl_nvtot its vacancy count.
template <int NW>
__device__ uint64_t sl_sector(StepShared& S, const Dyn& D, const Tables* tab, uint32_t k, int sid, int Sc,
                              double T) {
    constexpr int NT = NW * 32;
    const int tid = threadIdx.x;
    if (tid == 0) {
        const int ns = S.v.L / Sc, h = Sc / 2, oct = (int)(k & 7u);
        S.sl_h = h;
        S.sl_x0 = (sid % ns) * Sc + (oct & 1) * h;
        S.sl_y0 = ((sid / ns) % ns) * Sc + ((oct >> 1) & 1) * h;
        S.sl_z0 = (sid / (ns * ns)) * Sc + ((oct >> 2) & 1) * h;
    }
    __syncthreads();
    const int L = S.v.L;
    if (tid < 32) {
        const int nv = S.sl_nvtot;
        int n = 0;
        for (int b = 0; b < nv; b += 32) {
            const int q = b + tid;
            bool in = false;
            if (q < nv) {
                const int s = __ldcg(S.v.vac_pos + q), c = s >> 1, bit = s & 1;
                const int X = 2 * (c % L) + bit, Y = 2 * ((c / L) % L) + bit, Z = 2 * (c / (L * L)) + bit;
                in = sl_inside(S, X, Y, Z);
                D.apos[q] = X | (Y << 10) | (Z << 20);
            }
            const unsigned m = __ballot_sync(0xffffffffu, in);
            const int j = n + __popc(m & ((1u << tid) - 1u));
            if (in) D.gslot[j] = q;
            if (q < nv) D.lmap[q] = in ? j : -1;
            n += __popc(m);
        }
        if (tid == 0) S.sl_n = n;
    }
    __syncthreads();
    const int n_act = S.sl_n;
    if (n_act == 0) return 0;   // uniform
    load_tables<NW>(S, tab, S.v.model, 0);
    if (!S.sl_etab) {   // uniform
        for (int i = tid; i < kEtab; i += NT) D.etab[i] = S.v.etab[i];
    }
    int P = 1;
    while (P < n_act) P <<= 1;
    for (int j = tid; j < n_act; j += NT) {
        const int q = D.gslot[j], s = __ldcg(S.v.vac_pos + q), c = s >> 1, bit = s & 1;
        D.pos[j] = s;
        D.X[j] = 2 * (c % L) + bit;
        D.Y[j] = 2 * ((c / L) % L) + bit;
        D.Z[j] = 2 * (c / (L * L)) + bit;
        D.disp[3 * j + 0] = __ldcg(S.v.vac_disp + 3 * q + 0);
        D.disp[3 * j + 1] = __ldcg(S.v.vac_disp + 3 * q + 1);
        D.disp[3 * j + 2] = __ldcg(S.v.vac_disp + 3 * q + 2);
        D.on[j] = 1;
        D.fr[j] = !__ldcg(S.sl_stale + q);
    }
    for (int i = tid; i < 2 * P; i += NT) D.tree[i] = 0.0;
    __syncthreads();
    // vacancies whose stored rates are current: rates, sums and leaf from memory
    for (int i = tid; i < 8 * n_act; i += NT) {
        const int j = i >> 3, q = D.gslot[j];
        if (!D.fr[j]) continue;
        D.rates[i] = __ldcg(S.v.rates + 8 * q + (i & 7));
        D.dE[i] = __ldcg(S.v.dE + 8 * q + (i & 7));
        D.hop_sp[i] = __ldcg(S.v.hop_sp + 8 * q + (i & 7));
    }
    __syncthreads();
    for (int j = tid; j < n_act; j += NT) {
        if (!D.fr[j]) continue;
        const double* g = D.rates + 8 * j;
        double* h = D.hsum + 8 * j;
        h[4] = g[0] + g[1];
        h[5] = g[2] + g[3];
        h[6] = g[4] + g[5];
        h[7] = g[6] + g[7];
        h[2] = h[4] + h[5];
        h[3] = h[6] + h[7];
        h[1] = h[2] + h[3];
        D.tree[P + j] = h[1];
    }
    __syncthreads();
    if (tid == 0) {
        S.sl_etab = 1;
        S.v.nv = n_act;
        S.v.P = P;
        S.sl_k = (int32_t)k;
        S.sl_sid = sid;
        S.sl_t = 0.0;
        S.sl_T = T;
        S.n = 0;
        S.stop = 0;
        S.numeric = 0;
        S.ccount = 0;
        S.n_aff = 0;
        next_uniforms(S);
    }
    __syncthreads();
    const int mode = S.v.model == 0 ? 0 : (S.v.precision == 1 ? 1 : 2);
    for (int j = 0; j < n_act; ++j) {
        if (D.fr[j]) continue;   // uniform
        if (mode == 0)
            refresh_full<NW, 0>(S, D, j);
        else if (mode == 1)
            refresh_full<NW, 1>(S, D, j);
        else
            refresh_full<NW, 2>(S, D, j);
    }
    // inner nodes from the final leaves, level by level (each node = left + right)
    if (tid < 32) {
        for (int lv = P >> 1; lv >= 1; lv >>= 1) {
            for (int n = lv + tid; n < 2 * lv; n += 32) D.tree[n] = D.tree[2 * n] + D.tree[2 * n + 1];
            __syncwarp();
        }
    }
    __syncthreads();
    if (mode == 0)
        run_events_sl<NW, 0>(S, D);
    else if (mode == 1)
        run_events_sl<NW, 1>(S, D);
    else
        run_events_sl<NW, 2>(S, D);
    // the vacancies still inside the octant have current rates (refreshed after
    // every hop that could change them); those that left it may not
    for (int j = tid; j < n_act; j += NT) {
        const int q = D.gslot[j];
        S.v.vac_pos[q] = D.pos[j];
        S.v.vac_disp[3 * q + 0] = D.disp[3 * j + 0];
        S.v.vac_disp[3 * q + 1] = D.disp[3 * j + 1];
        S.v.vac_disp[3 * q + 2] = D.disp[3 * j + 2];
        S.sl_stale[q] = D.on[j] ? 0 : 1;
    }
    for (int i = tid; i < 8 * n_act; i += NT) {
        const int q = D.gslot[i >> 3];
        if (!D.on[i >> 3]) continue;
        S.v.rates[8 * q + (i & 7)] = D.rates[i];
        S.v.dE[8 * q + (i & 7)] = D.dE[i];
        S.v.hop_sp[8 * q + (i & 7)] = D.hop_sp[i];
    }
    return S.n;
}

// Voxel state for the sublattice kernels: the voxel record, no event log,
// L2-only lattice loads; stale[q] != 0 marks vacancy q's stored rates (rates,
// dE, hop species in the voxel record) as out of date.  Returns false
// (uniform) if the voxel is not OK.
template <int NW>
__device__ bool sl_begin(StepShared& S, const BatchArgs& a, int vid, int32_t* stale) {
    load_model<NW>(S, a.model);
    if (threadIdx.x == 0) {
        S.v = a.vox[vid];
        S.sl_nvtot = S.v.nv;
        S.v.log_cap = 0;
        S.sl_on = 1;
        S.sl_etab = 0;
        S.sl_stale = stale;
    }
    __syncthreads();
    return S.v.status == kOK;
}

__device__ __forceinline__ void sl_clock(VoxelDev* gv, double t_hi, double t_lo, double dt, uint32_t n) {
    for (uint32_t i = 0; i < n; ++i) {
        const double hi = t_hi + dt;
        if (fabs(t_hi) >= fabs(dt))
            t_lo += (t_hi - hi) + dt;
        else
            t_lo += (dt - hi) + t_hi;
        t_hi = hi;
    }
    gv->t_hi = t_hi;
    gv->t_lo = t_lo;
}

// Synchronous form: superstep k of voxel `vid`, one CTA per sector (grid
// (L/Sc)^3); the kernel boundary is the global barrier between supersteps.
template <int NW>
__global__ void __launch_bounds__(NW * 32) sl_kernel(BatchArgs a, int vid, uint32_t k, int Sc, double T,
                                                     int32_t* stale) {
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    __shared__ StepShared S;
    const Dyn D = carve(dyn_raw, a.max_nv, a.max_P, 0);
    VoxelDev* gv = &a.vox[vid];
    if (!sl_begin<NW>(S, a, vid, stale)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) sl_clock(gv, S.v.t_hi, S.v.t_lo, T * 0.125, 1);
    const uint64_t made = sl_sector<NW>(S, D, a.tab, k, blockIdx.x, Sc, T);
    if (threadIdx.x == 0) {
        if (made) atomicAdd((unsigned long long*)&gv->n_events, (unsigned long long)made);
        if (S.v.status != kOK) atomicCAS(&gv->status, kOK, S.v.status);
    }
}

// Asynchronous form (the readiness scheme of the sublattice method): one
// cooperative launch runs all n supersteps; CTA c owns sectors c, c + G, ...
// and takes its tasks (superstep i, sector) in superstep order.  done[s] = i
// records that sector s has finished supersteps < i; sector s starts
// superstep i once its 26 neighbours have done[.] >= i -- the only sectors
// whose superstep i - 1 can touch what superstep i of s reads or writes.
// Neighbouring sectors thus run the same superstep concurrently and never
// different ones, so the result equals the synchronous schedule; distant
// sectors drift apart freely.  All CTAs are resident (cooperative launch),
// and the smallest unfinished task always has its inputs ready, so the waits
// end; each wait is still bounded (a few seconds), after which the voxel gets
// kETIMEOUT and every CTA leaves at its next wait.  skip_sector >= 0 (a test
// hook) names a sector that is never processed nor reported, so that its
// neighbours' waits run out.
__device__ __forceinline__ int ld_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int32_t* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Warp 0: wait until the 26 neighbours of sector sid have done >= need.
// Returns false (to lane 0..31) on abort or timeout.
__device__ bool sl_wait(const int32_t* done, int32_t* abort_flag, int sid, int ns, int need, VoxelDev* gv) {
    const int lane = threadIdx.x & 31;
    int nb = sid;
    if (lane < 27 && lane != 13) {
        const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
        const int sx = sid % ns, sy = (sid / ns) % ns, sz = sid / (ns * ns);
        nb = (((sz + dz + ns) % ns) * ns + (sy + dy + ns) % ns) * ns + (sx + dx + ns) % ns;
    }
    for (int it = 0; it < (1 << 22); ++it) {
        const bool ok = ld_acquire(done + nb) >= need || nb == sid;
        const int ab = lane == 0 ? ld_acquire(abort_flag) : 0;
        if (__shfl_sync(0xffffffffu, ab, 0)) return false;
        if (__all_sync(0xffffffffu, ok)) return true;
        __nanosleep(200);
    }
    if (lane == 0) {
        atomicExch(abort_flag, 1);
        atomicCAS(&gv->status, kOK, kETIMEOUT);
    }
    return false;
}

template <int NW>
__global__ void __launch_bounds__(NW * 32) sl_async_kernel(BatchArgs a, int vid, uint32_t k0, uint32_t n, int Sc,
                                                           double T, int32_t* done, int32_t* abort_flag,
                                                           int32_t* stale, int skip_sector) {
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    __shared__ StepShared S;
    __shared__ int go;
    const Dyn D = carve(dyn_raw, a.max_nv, a.max_P, 0);
    VoxelDev* gv = &a.vox[vid];
    if (!sl_begin<NW>(S, a, vid, stale)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) sl_clock(gv, S.v.t_hi, S.v.t_lo, T * 0.125, n);
    const int ns = S.v.L / Sc, n_sec = ns * ns * ns;
    uint64_t made = 0;
    for (uint32_t i = 0; i < n; ++i) {
        for (int sid = blockIdx.x; sid < n_sec; sid += gridDim.x) {
            if (sid == skip_sector) continue;   // uniform
            if (threadIdx.x < 32) {
                const bool ok = sl_wait(done, abort_flag, sid, ns, (int)i, gv);
                if (threadIdx.x == 0) go = ok;
            }
            __syncthreads();
            if (!go) goto out;   // uniform
            made += sl_sector<NW>(S, D, a.tab, k0 + i, sid, Sc, T);
            // every thread's writes precede the barrier; thread 0's release store
            // (cumulative over them) publishes the sector's progress
            __syncthreads();
            if (threadIdx.x == 0) {
                if (S.v.status != kOK) {
                    atomicCAS(&gv->status, kOK, S.v.status);
                    atomicExch(abort_flag, 1);
                }
                st_release(done + sid, (int)i + 1);
            }
            if (S.v.status != kOK) goto out;   // uniform
        }
    }
out:
    if (threadIdx.x == 0 && made) atomicAdd((unsigned long long*)&gv->n_events, (unsigned long long)made);
}

// Full rebuild of one voxel per CTA: every vacancy's rates, then the tree
// (leaf path updates in slot order leave every node = left + right of its
// final children).
template <int NW>
__global__ void __launch_bounds__(NW * 32) rebuild_kernel(BatchArgs a, const int32_t* list) {
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    __shared__ StepShared S;
    const Dyn D = carve(dyn_raw, a.max_nv, a.max_P, 0);
    const int vid = list ? list[blockIdx.x] : (int)blockIdx.x;
    load_model<NW>(S, a.model);
    if (threadIdx.x == 0) S.v = a.vox[vid];
    __syncthreads();
    if (S.v.status == kEINVAL) return;   // placement failed; uniform
    load_tables<NW>(S, a.tab, S.v.model, S.v.L == 4);
    load_voxel_state<NW>(S, D);
    for (int i = threadIdx.x; i < 2 * S.v.P; i += NW * 32) D.tree[i] = 0.0;
    __syncthreads();
    const int mode = S.v.model == 0 ? 0 : (S.v.precision == 1 ? 1 : 2);
    for (int q = 0; q < S.v.nv; ++q) {
        if (mode == 0)
            refresh_full<NW, 0>(S, D, q);
        else if (mode == 1)
            refresh_full<NW, 1>(S, D, q);
        else
            refresh_full<NW, 2>(S, D, q);
    }
    if (threadIdx.x == 0 && S.numeric) S.v.status = kENUMERIC;
    __syncthreads();
    store_voxel_state<NW>(S, D, &a.vox[vid]);
}

// Per-voxel rate tables (see kEtab); etab_ok = 0 if any entry over- or underflows.
__global__ void rate_table_kernel(VoxelDev* vox, const ModelDev* M, const int32_t* list) {
    __shared__ int ok;
    VoxelDev& V = vox[list ? list[blockIdx.x] : (int)blockIdx.x];
    if (threadIdx.x == 0) ok = 1;
    __syncthreads();
    for (int i = threadIdx.x; i < kEtab; i += blockDim.x) {
        double v;
        if (i < 1536) {
            const int k = i >> 9, idx = i & 511;
            const double y = (double)idx * ldexp(1.0, 9 * k - 25);
            v = exp(-(V.beta * y));
        } else {
            v = M->nu * exp(V.beta * (2.0 - M->E0[i - 1536]));
        }
        V.etab[i] = v;
        if (!isfinite(v) || !(v >= 2.2250738585072014e-308)) ok = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) V.etab_ok = ok;
}

template <int NW>
static cudaError_t set_smem(const void* fn, size_t dyn) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

cudaError_t launch_rate_tables(VoxelDev* vox, int n_vox, const ModelDev* M, const int32_t* list,
                               cudaStream_t st) {
    rate_table_kernel<<<n_vox, 256, 0, st>>>(vox, M, list);
    return cudaGetLastError();
}

// The dynamic shared-memory attribute of step_kernel<warps> must have been set
// by step_occupancy() for this batch shape (no runtime call other than the
// launch happens here, so the launch can be captured in a CUDA graph).
cudaError_t launch_step(const BatchArgs& a, int warps, int grid, cudaStream_t st) {
    size_t dyn = step_dyn_smem(a.max_nv, a.max_P, a.win);
    switch (warps) {
#define AKMC_CASE(W)                                                              \
    case W:                                                                       \
        step_kernel<W><<<grid, W * 32, dyn, st>>>(a);                             \
        break;
        AKMC_CASE(1) AKMC_CASE(2) AKMC_CASE(4) AKMC_CASE(8) AKMC_CASE(16)
#undef AKMC_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rebuild(const BatchArgs& a, int warps, const int32_t* list, int n_list, cudaStream_t st) {
    const int grid = list ? n_list : a.n_vox;
    if (grid == 0) return cudaSuccess;
    size_t dyn = step_dyn_smem(a.max_nv, a.max_P, 0);
    cudaError_t e = cudaSuccess;
    switch (warps) {
#define AKMC_CASE(W)                                                              \
    case W:                                                                       \
        e = set_smem<W>((const void*)rebuild_kernel<W>, dyn);                     \
        if (e != cudaSuccess) return e;                                           \
        rebuild_kernel<W><<<grid, W * 32, dyn, st>>>(a, list);                    \
        break;
        AKMC_CASE(1) AKMC_CASE(2) AKMC_CASE(4) AKMC_CASE(8) AKMC_CASE(16)
#undef AKMC_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t sl_prepare(const BatchArgs& a) {
    return set_smem<8>((const void*)sl_kernel<8>, step_dyn_smem(a.max_nv, a.max_P, 0));
}

cudaError_t launch_sublattice(const BatchArgs& a, int vid, uint32_t k, int sector_cells, int n_sectors,
                              double window, int32_t* stale, cudaStream_t st) {
    sl_kernel<8><<<n_sectors, 256, step_dyn_smem(a.max_nv, a.max_P, 0), st>>>(a, vid, k, sector_cells, window,
                                                                             stale);
    return cudaGetLastError();
}

cudaError_t launch_sublattice_async(const BatchArgs& a, int vid, uint32_t k0, uint32_t n, int sector_cells,
                                    int n_sectors, double window, int32_t* done, int32_t* abort_flag,
                                    int32_t* stale, int skip_sector, int n_sm, int* grid_out, cudaStream_t st) {
    const size_t dyn = step_dyn_smem(a.max_nv, a.max_P, 0);
    cudaError_t e = set_smem<8>((const void*)sl_async_kernel<8>, dyn);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sl_async_kernel<8>, 256, dyn);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = std::min(n_sectors, per_sm * n_sm);
    *grid_out = grid;
    void* args[] = {(void*)&a,      (void*)&vid,    (void*)&k0,         (void*)&n,
                    (void*)&sector_cells, (void*)&window, (void*)&done, (void*)&abort_flag,
                    (void*)&stale,  (void*)&skip_sector};
    return cudaLaunchCooperativeKernel((const void*)sl_async_kernel<8>, dim3(grid), dim3(256), args, dyn, st);
}

// The dynamic shared-memory attribute only ever grows (per device and kernel),
// so a launch of one batch never runs with a limit set for a smaller one.
static std::mutex g_attr_mu;
static size_t g_attr_max[64][17];

int step_occupancy(int warps, int max_nv, int max_P, int win) {
    const size_t dyn = step_dyn_smem(max_nv, max_P, win);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || warps < 1 || warps > 16) return 0;
    {
        std::lock_guard<std::mutex> lock(g_attr_mu);
        size_t& cur = g_attr_max[dev][warps];
        if (dyn > cur) {
            const void* fn = warps == 1 ? (const void*)step_kernel<1> : warps == 2 ? (const void*)step_kernel<2>
                           : warps == 4 ? (const void*)step_kernel<4> : warps == 8 ? (const void*)step_kernel<8>
                           : (const void*)step_kernel<16>;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
                return 0;
            cur = dyn;
        }
    }
    int n = 0;
    switch (warps) {
        case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<1>, 32, dyn); break;
        case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<2>, 64, dyn); break;
        case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<4>, 128, dyn); break;
        case 8: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<8>, 256, dyn); break;
        case 16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<16>, 512, dyn); break;
        default: break;
    }
    return n;
}

}  // namespace akmc
