// akmc_device.cuh -- device-side layout and helpers shared by the kernels of
// libakmc (the GB300 vacancy AKMC library).  Everything a kernel needs lives in
// the caller's workspace; the structs below describe that memory.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace akmc {

constexpr int kFe = 0, kVac = 4;
constexpr int kRhoBits = 24;          // density fixed point: units of 2^-24
constexpr int kEBits = 40;            // split-mode energy fixed point: units of 2^-40 eV
constexpr int kPairU = 59;            // sites read to rate all 8 hops, pair model
constexpr int kPairE = 26;            // terms per hop, pair model (13 bonds of w, 13 of m)
constexpr int kEamU = 145;            // sites read to rate all 8 hops, EAM
constexpr int kEamE = 77;             // 76 neighbour terms + the moving atom's own term
constexpr int kSph = 58;              // sites within the EAM cutoff (shells 1..5)
constexpr int kMaxNV = 256;
constexpr double kKB = 8.617333262e-5;   // eV/K

enum Status { kOK = 0, kEINVAL = 1, kENOMEM = 2, kECUDA = 3, kETIMEOUT = 4, kETRAPPED = 5, kENUMERIC = 6 };

// F_k and the Horner coefficients of one embedding interval (FP64).
struct __align__(32) Cubic64 { double F, c1, c2, c3; };

// Half-unit offset packed in an int32: bits [0,6) dx+16, [6,12) dy+16,
// [12,18) dz+16, bits 18+ an extra field (shell number, ...).
__host__ __device__ __forceinline__ int32_t off_pack(int dx, int dy, int dz, int extra) {
    return (dx + 16) | ((dy + 16) << 6) | ((dz + 16) << 12) | (extra << 18);
}
__host__ __device__ __forceinline__ int off_dx(int32_t o) { return (o & 63) - 16; }
__host__ __device__ __forceinline__ int off_dy(int32_t o) { return ((o >> 6) & 63) - 16; }
__host__ __device__ __forceinline__ int off_dz(int32_t o) { return ((o >> 12) & 63) - 16; }
__host__ __device__ __forceinline__ int off_extra(int32_t o) { return o >> 18; }

// Stencil tables (built on the host once, stored in the workspace).
struct Tables {
    int32_t pair_off[64];      // union stencil of the pair model; [0] = the vacancy itself
    int32_t pair_mk[8];        // union index of hop target m_k
    uint32_t pair_ent[8][32];  // per hop: idx | (shell-1)<<8 | side<<9  (side 1: bond of m)
    int32_t eam_off[160];      // union stencil of EAM; [0] = the vacancy itself
    int32_t eam_mk[8];
    uint32_t eam_ent[8][80];   // idx | s_ip<<8 | s_im<<11 | own<<14   (shell 0 = outside)
    int32_t sph_off[64];       // the 58 cutoff-sphere offsets, extra = shell
    // For the EAM union stencil around a vacancy that has just moved from w
    // to m = w + d_k (entry u at offset o_u from m): (shell(u - w) << 3) |
    // shell(u - m), the shells of the density change f_A(r_uw) - f_A(r_um)
    // that the hop caused at u.  [0]: L >= 5; [1]: L = 4 (u - w taken as the
    // periodic minimal image).
    uint8_t eam_dsh[2][160][8];
    // Prefetch region of a single vacancy at p: the union of the read sets of
    // all 8 possible next positions p + d_k (offsets relative to p), and, per
    // hop direction d, the region index of every union entry around p + d.
    int32_t pair_roff[160];
    uint16_t pair_ridx[8][64];
    int32_t eam_roff[288];
    uint16_t eam_ridx[8][160];
    int32_t pair_nreg, eam_nreg;
    int32_t pair_rc[9], eam_rc[9];   // region index of p itself ([8]) and of p + d_k ([k])
};

struct ModelDev {
    int32_t eps_q[2][25];      // pair energies in units of 2^-24 eV
    double E0[4];
    double nu;
    double a, r_cut, rho_h, inv_knot;   // inv_knot = 2^-shift
    int32_t n_r, n_rho, shift, has_eam;
    int32_t thr_hi[4];         // dE_q > thr_hi[A]  <=>  dE > 2 E0[A]   (dE_q in units of 2^-24 eV)
    int32_t thr_lo[4];         // dE_q < thr_lo[A]  <=>  dE < -2 E0[A]
    double two_E0[4];
    int32_t rho_pure;          // perfect-Fe density (fixed point)
    int32_t rho_max;           // largest density any site can reach (fixed point)
    int32_t fq[5][8];          // density contribution f_b(shell), row V = 0, shell 0 = 0
    int32_t cq[5][8];          // fq[b] - fq[Fe]: correction to the perfect-Fe density
    double phi_d[10][8];       // phi_ab(shell) in eV, shell 0 = 0
    long long phi_q[10][8];    // same in units of 2^-40 eV
    const double* phi_tab;     // raw tables (workspace copies)
    const double* f_tab;
    const double* F_tab;
    Cubic64* Fd;               // [4][n_rho-1]: F_k, c1, c2, c3 (FP64 Horner in t)
    float4* Ff;                // [4][n_rho]: c1, c2, c3, 0 (FP32); the last knot of each species is all zero
    long long* Fq;             // [4][n_rho]: F_k in units of 2^-40 eV
};

struct VoxelDev {
    int32_t L, N, nv, P;       // P = next power of two >= nv
    int32_t model, precision, status, log_cap;
    int32_t counts[4];         // vacancies, Cu, Ni, Mn
    double beta;               // 1/(kB T)
    double frac[3];
    double T;
    uint64_t seed, uid;
    uint64_t n_events;
    double t_hi, t_lo;
    uint8_t* species;
    int32_t* rho;              // EAM only
    int32_t* vac_pos;
    int32_t* vac_disp;         // [3 nv]
    double* rates;             // [8 nv]
    double* dE;                // [8 nv]
    double* tree;              // [2P], node 1 = root
    uint8_t* hop_sp;           // [8 nv] species at each hop target
    int32_t* log;              // [log_cap]
    double* etab;              // [kEtab] rate tables of this temperature (see kEtab)
    int32_t etab_ok;           // tables finite and nonzero (else rates use exp directly)
    int32_t pad_;
};

// Per-voxel rate tables: exp(-beta * i * 2^(9k) * 2^-25) for k = 0,1,2 and
// i < 512 (energies on the 2^-25 eV grid below 4 eV), then for each jumping
// species A the constant nu * exp(beta * (2 - E0[A])).
constexpr int kEtab = 3 * 512 + 4;

struct BatchArgs {
    VoxelDev* vox;
    const ModelDev* model;
    const Tables* tab;
    const int32_t* order;      // processing order of voxels
    const uint64_t* targets;   // events to run this call, per voxel
    uint32_t* queue;           // persistent work-queue head
    int32_t* batch_status;     // batch-level error word
    int32_t n_vox;
    int32_t max_nv, max_P;
    int32_t win;               // edge (cells) of the shared-memory lattice window, 0 = none
};

// Edge (cells) of the shared-memory lattice window of a single-vacancy voxel.
// The window path steps single-vacancy voxels of the pair model or of EAM in
// split precision with L >= 5 (the stencils of the vacancy and of its 8
// targets fit in a window of min(L, 16) cells with no periodic self-aliasing).
constexpr int kWinMax = 16;
__host__ __device__ inline int window_edge(int L, int n_vac, int model, int precision) {
    if (n_vac != 1 || L < 5 || (model != 0 && precision != 1)) return 0;
    return L < kWinMax ? L : kWinMax;
}

// ---------------------------------------------------------------- helpers

__host__ __device__ __forceinline__ int pair_index(int a, int b) {
    if (a > b) { int t = a; a = b; b = t; }
    return a * (7 - a) / 2 + b;
}

__device__ __forceinline__ int wrap_coord(int X, int M) {   // X in [-M, 2M)
    X = X < 0 ? X + M : X;
    return X >= M ? X - M : X;
}

__device__ __forceinline__ int site_index(int X, int Y, int Z, int L) {
    return ((((Z >> 1) * L + (Y >> 1)) * L + (X >> 1)) << 1) | (X & 1);
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products
// with Weyl-sequence key bumps between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
}

// Uniforms of event n of a voxel: counter (n_lo, n_hi, uid_lo, uid_hi & 0x7fffffff),
// key (seed_lo, seed_hi); u1 in [0,1), u2 in (0,1], 53 bits each.
__device__ __forceinline__ void event_uniforms(uint64_t seed, uint64_t uid, uint64_t n,
                                               double& u1, double& u2) {
    uint32_t c0 = (uint32_t)n, c1 = (uint32_t)(n >> 32), c2 = (uint32_t)uid,
             c3 = (uint32_t)(uid >> 32) & 0x7fffffffu;
    philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    uint64_t a = ((uint64_t)c0 << 21) | (c1 >> 11);
    uint64_t b = ((uint64_t)c2 << 21) | (c3 >> 11);
    u1 = (double)a * 0x1p-53;
    u2 = (double)(b + 1) * 0x1p-53;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

}  // namespace akmc
