// k_density.cu -- EAM site densities from the lattice (build_density):
//   rho_i = sum_{j in S(i), s_j != V} f_{s_j}(r_ij)   (fixed point, exact).
//
// Two kernels.  Voxels with L <= 256 use the strip kernel (below): full
// x-rows streamed along z, 16-byte loads and stores.  Larger voxels use the
// tile kernel: a streaming stencil over tiles of 32 x 16 x 16 cells.  A perfect-Fe lattice
// has the same density everywhere, so each tile starts from that value in
// shared memory and only the non-Fe sites of the haloed tile (solutes and
// vacancies, a few percent) scatter their corrections f_s - f_Fe to their 58
// neighbours with shared-memory atomics (integer, hence order-independent).
// Global traffic is one read of the haloed species tile (row by row, one
// 32-byte sector per warp access) and one coalesced write of the density
// tile.  The non-Fe sites of each slab of halo rows are first compacted into
// a list (ballot, one append per warp), then one warp per listed site adds
// its 58 corrections (distinct targets, so lanes never conflict).
#include "akmc_device.cuh"
#include "akmc_launch.h"

#include <utility>

namespace akmc {

constexpr int kDensThreads = 256;
constexpr int kDensWarps = kDensThreads / 32;
constexpr int kSlabRows = 64;                                   // halo rows compacted per pass
constexpr int kListCap = kSlabRows * 2 * (kTX + 2 * kHalo);     // every site of a slab

__global__ void __launch_bounds__(kDensThreads) density_tile_kernel(const VoxelDev* vox, const ModelDev* M,
                                                               const Tables* tab, const int4* items) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int32_t s_off[64];
    __shared__ int32_t s_cq[5][8];
    __shared__ uint16_t s_list[kListCap];
    __shared__ int s_nlist;
    const int4 it = items[blockIdx.x];
    const VoxelDev& V = vox[it.x];
    const int L = V.L;
    const int x0 = it.y, y0 = it.z, z0 = it.w;
    const int tx = min(kTX, L - x0), ty = min(kTY, L - y0), tz = min(kTZ, L - z0);
    const int hx = tx + 2 * kHalo, hy = ty + 2 * kHalo, hz = tz + 2 * kHalo;
    const int hrow = 2 * hx, trow = 2 * tx;               // bytes per halo row, sites per tile row
    int32_t* rt = (int32_t*)sm;                           // [tz][ty][2 tx]
    uint8_t* hs = sm + sizeof(int32_t) * kTX * kTY * kTZ * 2;   // [hz][hy][2 hx]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kSph) s_off[tid] = tab->sph_off[tid];
    if (tid < 40) s_cq[tid / 8][tid % 8] = M->cq[tid / 8][tid % 8];
    if (tid == 0) s_nlist = 0;
    const int32_t rho0 = M->rho_pure;
    const uint8_t* sp = V.species;
    // haloed species tile, one row (fixed y, z) per warp iteration
    for (int r = warp; r < hz * hy; r += kDensWarps) {
        int y = y0 - kHalo + r % hy, z = z0 - kHalo + r / hy;
        y = y < 0 ? y + L : (y >= L ? y - L : y);
        z = z < 0 ? z + L : (z >= L ? z - L : z);
        const uint8_t* row = sp + ((size_t)z * L + y) * L * 2;
        uint8_t* dst = hs + r * hrow;
        for (int c = lane; c < hrow; c += 32) {
            int x = x0 - kHalo + (c >> 1);
            x = x < 0 ? x + L : (x >= L ? x - L : x);
            dst[c] = row[2 * x + (c & 1)];
        }
    }
    for (int i = tid; i < tz * ty * trow; i += kDensThreads) rt[i] = rho0;
    __syncthreads();
    const int n_rows = hz * hy;
    for (int r0 = 0; r0 < n_rows; r0 += kSlabRows) {
        const int r1 = min(n_rows, r0 + kSlabRows);
        for (int r = r0 + warp; r < r1; r += kDensWarps) {
            const uint8_t* src = hs + r * hrow;
            for (int c0 = 0; c0 < hrow; c0 += 32) {
                const int c = c0 + lane;
                const bool hit = c < hrow && src[c] != kFe;
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                int base = 0;
                if (lane == 0 && m) base = atomicAdd(&s_nlist, __popc(m));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (hit) s_list[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)((r - r0) * hrow + c);
            }
        }
        __syncthreads();
        const int nl = s_nlist;
        for (int i = warp; i < nl; i += kDensWarps) {
            const int rel = s_list[i];
            const int rr = r0 + rel / hrow, c = rel % hrow;
            const int s = hs[rr * hrow + c];
            const int b = c & 1;
            const int HX = c, HY = 2 * (rr % hy) + b, HZ = 2 * (rr / hy) + b;   // half units, halo frame
            for (int k = lane; k < kSph; k += 32) {
                const int o = s_off[k];
                const int X = HX + off_dx(o), Y = HY + off_dy(o), Z = HZ + off_dz(o);
                if (X < 0 || Y < 0 || Z < 0) continue;
                const int ix = (X >> 1) - kHalo, iy = (Y >> 1) - kHalo, iz = (Z >> 1) - kHalo;
                if (ix < 0 || iy < 0 || iz < 0 || ix >= tx || iy >= ty || iz >= tz) continue;
                atomicAdd(&rt[(iz * ty + iy) * trow + 2 * ix + (X & 1)], s_cq[s][off_extra(o)]);
            }
        }
        __syncthreads();
        if (tid == 0) s_nlist = 0;
        __syncthreads();
    }
    // coalesced write of the density tile, one row per warp iteration
    int32_t* rho = V.rho;
    for (int r = warp; r < tz * ty; r += kDensWarps) {
        const int cy = r % ty, cz = r / ty;
        int32_t* dst = rho + (((size_t)(z0 + cz) * L + (y0 + cy)) * L + x0) * 2;
        const int32_t* src = rt + r * trow;
        for (int c = lane; c < trow; c += 32) dst[c] = src[c];
    }
}


// ---- strip kernel: full x-rows, streamed along z -----------------------------
// One CTA owns the rows y in [y0, y0+ty) of the planes z in [z0, z0+tz) of one
// voxel.  It walks the source planes z0-2 .. z0+tz+1 once, in blocks of 4.
// Per block:
//  a. append: the block's haloed strips (ty+4 rows of 2L sites per plane,
//     16-byte chunks, loaded one block ahead into registers) are scanned for
//     non-Fe bytes with a few word
//     operations per 4 sites; each non-Fe site becomes one list entry
//     (species, buffer position, halo row), in one list per sublattice
//     (b = X & 1): entries of the strip's own rows at the front, of the 2 + 2
//     halo rows at the back;
//  b. scatter (all warps): warps 0, 2, 4, 6 take the b = 0 list and warps
//     1, 3, 5, 7 the b = 1 list, 8 lanes per entry; a lane holds the
//     shared-memory byte deltas of its 8 stencil offsets for its warp's b
//     (registers) and fetches the entry species' weights f_s - f_Fe with two
//     16-byte loads, then adds them to a buffer of 8 density planes with
//     shared-memory reductions (integer, hence order-independent).  Every
//     plane has 2 guard rows on each side, so the strip's own rows need no
//     check; halo-row entries predicate each term on its target row;
//  c. pads: the row pads (4 sites on each side, so an x offset needs no wrap)
//     of buffer planes 0..3 are folded into the row ends, planes 4..7's pads
//     move down;
//  d. shift: planes 0..3 are complete and written with 16-byte stores (planes
//     outside the CTA's z range are dropped); planes 4..7 move down and
//     restart as pure Fe.  Four barriers per block.
// A block whose lists would overflow (a locally dense lattice, > 1024 entries
// of one sublattice) is scattered directly from memory instead, one site per
// thread (slow, exact).
//
// Site coordinates: within a row (fixed y, z) the site index 2x+b equals the
// half-unit coordinate X, so a neighbour at half-unit offset dx sits at
// X + dx (mod 2L) of the row that holds cell floor((Y + dy)/2).
//
// Per output site the work is one species byte read, one density write and,
// for the ~2% non-Fe sites (x the halo factor (ty+4)/ty * (tz+4)/tz), 58
// shared-memory reductions.

constexpr int kStripThreads = 256;
constexpr int kBlk = 4;             // source planes per block
constexpr int kPlanes = kBlk + 4;   // density planes held
constexpr int kRowPad = 4;          // padding sites on each side of a buffer row
constexpr int kGuard = 2;           // guard rows on each side of a buffer plane
constexpr int kChunks = 3;          // 16-byte chunks per thread and block (host-guaranteed)
constexpr int kStripCap = 1024;     // entries per sublattice list and block
constexpr int kOffs = 8;            // stencil offsets per scatter lane: k = sub + 8j

__host__ __device__ inline int strip_rw(int L) { return 2 * L + 2 * kRowPad; }
__host__ __device__ inline int strip_slot(int TY, int L) { return (TY + 2 * kGuard) * strip_rw(L) + 4; }
// buffer planes and two lists
__host__ __device__ inline size_t strip_smem(int TY, int L) {
    return sizeof(int32_t) * ((size_t)kPlanes * strip_slot(TY, L) + 2 * (size_t)kStripCap);
}
// rows per strip: 16 for L <= 64, 8 for L <= 128, 2 beyond (shared memory and kChunks)
__host__ __device__ inline int strip_rows(int L) { return L <= 64 ? 16 : (L <= 128 ? 8 : 2); }
// edge of the fixed buffer geometry of the 16-byte path (L <= 128)
__host__ __device__ inline int strip_geom_L(int L) { return L <= 32 ? 32 : (L <= 64 ? 64 : 128); }

// floor((b + d) / 2) for b in {0,1}, d in [-4, 4]
__device__ __forceinline__ int half_floor(int v) { return (v + 8) / 2 - 4; }

// Bit j of the result: byte j of the 16-byte chunk is non-zero.
__device__ __forceinline__ uint32_t nonzero_bytes(uint4 v) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t M = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t t = (((w[i] & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w[i]) & 0x80808080u;   // bit 7 per byte
        M |= (((t >> 7) * 0x10204080u) >> 28) << (4 * i);                                 // bits 0, 8, 16, 24 -> 0..3
    }
    return M;
}

// Entry: species (3 bits, codes above 7 clamped) | buffer position u << 3 | halo row << 23,
// u = (plane in block + 2) * SLOT + hr * RW + X + kRowPad (halo row hr = buffer row).
__device__ __forceinline__ uint32_t strip_entry(uint32_t s, int u, int hr) {
    return (s > 7 ? 7u : s) | ((uint32_t)u << 3) | ((uint32_t)hr << 23);
}

// Halo rows hr in [2, ty+2) are the strip's own rows: every target lies in the buffer.
__device__ __forceinline__ bool strip_own(int hr, int ty) { return hr >= 2 && hr < ty + 2; }

__device__ __forceinline__ void strip_push(uint32_t* lists, uint32_t en, int b, bool own, int at) {
    if (at < kStripCap) lists[b * kStripCap + (own ? at : kStripCap - 1 - at)] = en;
}

// shared-memory reduction at byte address a; the predicated form adds iff row < ty
__device__ __forceinline__ void red_add(uint32_t a, int v) {
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_if(uint32_t a, int v, uint32_t row, uint32_t ty) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %2, %3;\n\t@p red.shared.add.s32 [%0], %1;\n\t}" ::"r"(a), "r"(v),
                 "r"(row), "r"(ty)
                 : "memory");
}

// Weight f_s - f_Fe of stencil offset k for species s (table [s][k & 7][k >> 3]).
__device__ __forceinline__ int strip_w(const int4 (*wt)[8][2], int s, int k) {
    return ((const int32_t*)wt)[s * 64 + (k & 7) * 8 + (k >> 3)];
}

template <bool VEC>
__device__ void strip_body(const VoxelDev& V, const int4 it, int32_t* buf, uint32_t* lists,
                           const int4 (*wt)[8][2], const int32_t* sph, int* cnt, int32_t rho0) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = V.L, M2 = 2 * L;
    const int y0 = it.y, z0 = it.z, tz = it.w & 0xFFFF, TY = it.w >> 17;
    const int ty = min(TY, L - y0);
    const int RW = strip_rw(L), SLOT = strip_slot(TY, L);
    const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(buf);
    // this lane's stencil offsets k = sub + 8j for sublattice b = warp & 1:
    // byte delta 4 (dzc*SLOT + dyc*RW + dx) and, 3 bits each, dyc + 2
    const int sub = lane & 7, b = warp & 1;
    int Dl[kOffs];
    uint32_t DY = 0;
#pragma unroll
    for (int j = 0; j < kOffs; ++j) {
        const int k = sub + 8 * j;
        const int o = k < kSph ? sph[k] : sph[0];
        const int dyc = half_floor(b + off_dy(o)), dzc = half_floor(b + off_dz(o));
        Dl[j] = 4 * (dzc * SLOT + dyc * RW + off_dx(o));
        DY |= (uint32_t)(dyc + 2) << (3 * j);
    }
    const uint32_t k7 = sub < kSph - 56 ? 0u : 1u;    // offset sub + 56 exists iff 0
    // buffer: planes qb .. qb+7 (relative plane index; rel. plane 2 is z0); the
    // strip's rows pure Fe, pads and guard rows 0
    for (int pr = warp; pr < kPlanes * (ty + 2 * kGuard); pr += kStripThreads / 32) {
        const int p = pr / (ty + 2 * kGuard), br = pr - p * (ty + 2 * kGuard);
        int32_t* row = buf + p * SLOT + br * RW;
        const bool own = br >= kGuard && br < ty + kGuard;
        for (int c = lane; c < RW; c += 32) row[c] = own && c >= kRowPad && c < kRowPad + M2 ? rho0 : 0;
    }
    // z and y indices in [-2, 2L) wrap with one correction
    auto wrap = [&](int z) { return z < 0 ? z + L : (z >= L ? z - L : z); };
    const int n_src = tz + 4;
    // this thread's chunks k: 16 sites of halo row hr_k of plane pl_k of a block
    // (the same for every block); off = offset of the chunk in its plane
    const int cpr = M2 / 16;                           // 16-byte chunks per row (VEC)
    const int per_plane = (ty + 4) * cpr;
    int ck_pl[kChunks], ck_hr[kChunks], ck_u[kChunks], ck_off[kChunks];
#pragma unroll
    for (int k = 0; k < kChunks; ++k) {
        const int c = tid + k * kStripThreads;
        const int pl = VEC ? c / per_plane : 0, rem = c - pl * per_plane;
        const int hr = VEC ? rem / cpr : 0, cx = rem - hr * cpr;
        ck_pl[k] = pl;
        ck_hr[k] = hr;
        ck_u[k] = (pl + 2) * SLOT + hr * RW + 16 * cx + kRowPad;
        ck_off[k] = wrap(y0 - 2 + hr) * M2 + 16 * cx;
    }
    uint4 v[kChunks];
    auto load_block = [&](int rb) {
        const int nb = min(kBlk, n_src - rb);
#pragma unroll
        for (int k = 0; k < kChunks; ++k)
            if (ck_pl[k] < nb)
                v[k] = __ldcs((const uint4*)(V.species + (size_t)wrap(z0 - 2 + rb + ck_pl[k]) * L * M2 + ck_off[k]));
    };
    if (VEC) load_block(0);
    if (tid < 4) cnt[tid] = 0;
    __syncthreads();
    int qb = -2;
    for (int rb = 0; rb < n_src; rb += kBlk, qb += kBlk) {
        const int nb = min(kBlk, n_src - rb);
        // a. append
        if (VEC) {
#pragma unroll
            for (int k = 0; k < kChunks; ++k) {
                if (ck_pl[k] >= nb) break;
                uint32_t M = nonzero_bytes(v[k]);
                if (!M) continue;
                const int hr = ck_hr[k];
                const bool own = strip_own(hr, ty);
                const uint32_t M0 = M & 0x5555u, M1 = M & 0xAAAAu;
                int a0 = M0 ? atomicAdd(&cnt[own ? 0 : 1], __popc(M0)) : 0;
                int a1 = M1 ? atomicAdd(&cnt[own ? 2 : 3], __popc(M1)) : 0;
                while (M) {
                    const int j = __ffs(M) - 1;
                    M &= M - 1;
                    const uint32_t wj = j < 8 ? (j < 4 ? v[k].x : v[k].y) : (j < 12 ? v[k].z : v[k].w);
                    const uint32_t en = strip_entry((wj >> (8 * (j & 3))) & 0xFFu, ck_u[k] + j, hr);
                    if (j & 1) strip_push(lists, en, 1, own, a1++);
                    else strip_push(lists, en, 0, own, a0++);
                }
            }
            if (rb + kBlk < n_src) load_block(rb + kBlk);   // next block, in flight during the scatter
        } else {
            const int n = nb * (ty + 4) * M2;
            for (int c = tid; c < n; c += kStripThreads) {
                const int pl = c / ((ty + 4) * M2), rem = c - pl * (ty + 4) * M2, hr = rem / M2, X = rem - hr * M2;
                const uint32_t sp = V.species[((size_t)wrap(z0 - 2 + rb + pl) * L + wrap(y0 - 2 + hr)) * M2 + X];
                if (sp != 0) {
                    const bool own = strip_own(hr, ty);
                    const int bb = X & 1;
                    const int at = atomicAdd(&cnt[2 * bb + (own ? 0 : 1)], 1);
                    strip_push(lists, strip_entry(sp, (pl + 2) * SLOT + hr * RW + X + kRowPad, hr), bb, own, at);
                }
            }
        }
        __syncthreads();
        // b. scatter
        const bool ovf = cnt[0] + cnt[1] > kStripCap || cnt[2] + cnt[3] > kStripCap;   // uniform
        if (!ovf) {
            const uint32_t* lst = lists + b * kStripCap;
            const int first = (warp >> 1) * 4 + (lane >> 3);   // 16 entries per pass and sublattice
            const int ni = cnt[2 * b], ne = cnt[2 * b + 1];
            for (int i = first; i < ni; i += 16) {
                const uint32_t en = lst[i];
                const uint32_t ub = sbuf + 4 * ((en >> 3) & 0xFFFFFu);
                const int4 w0 = wt[en & 7][sub][0], w1 = wt[en & 7][sub][1];
                const int ww[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                for (int j = 0; j < kOffs - 1; ++j) red_add(ub + Dl[j], ww[j]);
                red_add_if(ub + Dl[kOffs - 1], ww[kOffs - 1], k7, 1u);
            }
            for (int i = first; i < ne; i += 16) {
                const uint32_t en = lst[kStripCap - 1 - i];
                const uint32_t ub = sbuf + 4 * ((en >> 3) & 0xFFFFFu);
                const uint32_t hm = (en >> 23) - 4u;            // target row hr + dyc - 2 = hm + (dyc + 2)
                const int4 w0 = wt[en & 7][sub][0], w1 = wt[en & 7][sub][1];
                const int ww[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                for (int j = 0; j < kOffs; ++j) {
                    const uint32_t row = j == kOffs - 1 && k7 ? 0xFFFFFFFFu : hm + ((DY >> (3 * j)) & 7);
                    red_add_if(ub + Dl[j], ww[j], row, (uint32_t)ty);
                }
            }
        } else {
            // direct scatter of the block, one source site per thread and pass
            const int n = nb * (ty + 4) * M2;
            for (int c = tid; c < n; c += kStripThreads) {
                const int pl = c / ((ty + 4) * M2), rem = c - pl * (ty + 4) * M2, hr = rem / M2, X = rem - hr * M2;
                uint32_t sp = V.species[((size_t)wrap(z0 - 2 + rb + pl) * L + wrap(y0 - 2 + hr)) * M2 + X];
                if (sp == 0) continue;
                sp = sp > 7 ? 7 : sp;
                const int bb = X & 1, u = (pl + 2) * SLOT + hr * RW + X + kRowPad;
                for (int k = 0; k < kSph; ++k) {
                    const int o = sph[k];
                    const int dyc = half_floor(bb + off_dy(o)), dzc = half_floor(bb + off_dz(o));
                    if ((unsigned)(hr + dyc - 2) < (unsigned)ty)
                        atomicAdd(buf + u + dzc * SLOT + dyc * RW + off_dx(o), strip_w(wt, sp, k));
                }
            }
        }
        __syncthreads();
        // c. pads of planes 0..3 into their row ends; planes 4..7's pads move down
        for (int t = tid; t < kBlk * ty * 2; t += kStripThreads) {
            const int i = t / (2 * ty), rem = t - i * 2 * ty, r = rem >> 1;
            int32_t* row = buf + i * SLOT + (r + kGuard) * RW;
            int32_t* up = row + kBlk * SLOT;
            if ((rem & 1) == 0) {             // sites 0..2 collect the right pads (X = 2L .. 2L+2)
#pragma unroll
                for (int k = 0; k < 3; ++k) row[kRowPad + k] += row[kRowPad + M2 + k];
#pragma unroll
                for (int k = 0; k < kRowPad; ++k) {
                    row[kRowPad + M2 + k] = up[kRowPad + M2 + k];
                    up[kRowPad + M2 + k] = 0;
                }
            } else {                          // sites 2L-3..2L-1 collect the left pads (X = -3 .. -1)
#pragma unroll
                for (int k = 0; k < 3; ++k) row[kRowPad + M2 - 3 + k] += row[kRowPad - 3 + k];
#pragma unroll
                for (int k = 0; k < kRowPad; ++k) {
                    row[k] = up[k];
                    up[k] = 0;
                }
            }
        }
        __syncthreads();
        // d. shift: planes 0..3 are complete
        if (VEC) {
            const int4 pure = make_int4(rho0, rho0, rho0, rho0);
#pragma unroll
            for (int i = 0; i < kBlk; ++i) {
                const int q = qb + i;
                const bool wr = q >= 2 && q < tz + 2;
                int4* out = (int4*)(V.rho + ((size_t)(z0 + q - 2) * L + y0) * M2);
                for (int r = warp; r < ty; r += kStripThreads / 32) {
                    int4* row = (int4*)(buf + i * SLOT + (r + kGuard) * RW + kRowPad);
                    int4* up = (int4*)((int32_t*)row + kBlk * SLOT);
                    int4* orow = out + r * (M2 / 4);
                    for (int c = lane; c < M2 / 4; c += 32) {
                        const int4 val = row[c];
                        if (wr) __stcs(orow + c, val);
                        row[c] = up[c];
                        up[c] = pure;
                    }
                }
            }
        } else {
            for (int f = tid; f < kBlk * ty * M2; f += kStripThreads) {
                const int i = f / (ty * M2), rem = f - i * (ty * M2), r = rem / M2, X = rem - r * M2;
                int32_t* row = buf + i * SLOT + (r + kGuard) * RW + kRowPad;
                const int q = qb + i;
                if (q >= 2 && q < tz + 2) V.rho[((size_t)(z0 + q - 2) * L + y0 + r) * M2 + X] = row[X];
                row[X] = row[X + kBlk * SLOT];
                row[X + kBlk * SLOT] = rho0;
            }
        }
        if (tid < 4) cnt[tid] = 0;
        __syncthreads();
    }
}

// ---- fixed-geometry strip path (16-byte rows, L <= 128) ------------------------
// The same strip walk with the buffer geometry fixed at compile time (row
// stride 2 LG + 8, LG in {32, 64, 128} the smallest one >= L, TYG rows per
// strip), so every stencil offset is an immediate in the reduction's address.
// Scatter: one list entry per lane, 32 entries per warp pass; a lane adds its
// entry's 58 weights with 58 reductions at [entry + constant] (halo-row entries
// predicate each term on its target row).  Row pads fold into the row ends in
// the write-out itself, and the write-out of a block shares its phase with the
// list building of the next one: two CTA barriers per block of 4 planes.

// The 58 cutoff-sphere offsets (half units) and their shells, in a fixed order.
struct StencilTab {
    int dx[kSph], dy[kSph], dz[kSph], sh[kSph];
};
constexpr StencilTab make_stencil() {
    StencilTab t{};
    int n = 0;
    for (int dz = -3; dz <= 3; ++dz)
        for (int dy = -3; dy <= 3; ++dy)
            for (int dx = -3; dx <= 3; ++dx) {
                const int q = dx * dx + dy * dy + dz * dz;
                const int sh = q == 3 ? 1 : q == 4 ? 2 : q == 8 ? 3 : q == 11 ? 4 : q == 12 ? 5 : 0;
                if (sh == 0 || ((dx ^ dy) & 1) || ((dy ^ dz) & 1)) continue;
                t.dx[n] = dx, t.dy[n] = dy, t.dz[n] = dz, t.sh[n] = sh;
                ++n;
            }
    return t;
}
constexpr StencilTab kStencil = make_stencil();
constexpr int hfloor_c(int v) { return (v + 8) / 2 - 4; }
// Offset K seen from a sublattice-B site in a buffer of row stride RW and plane
// stride SLOT: its shell, its cell row offset and its buffer-word delta, all
// compile-time constants.
template <int B, int RW, int SLOT, int K>
struct StOff {
    static constexpr int sh = kStencil.sh[K];
    static constexpr int dyc = hfloor_c(B + kStencil.dy[K]);
    static constexpr int delta = hfloor_c(B + kStencil.dz[K]) * SLOT + dyc * RW + kStencil.dx[K];
};
template <int B, int RW, int SLOT>
constexpr int st_min_f() {
    int m = 0;
    for (int k = 0; k < kSph; ++k) {
        const int d = hfloor_c(B + kStencil.dz[k]) * SLOT + hfloor_c(B + kStencil.dy[k]) * RW + kStencil.dx[k];
        m = d < m ? d : m;
    }
    return m;
}
template <int B, int RW, int SLOT>
struct StMin {
    static constexpr int v = st_min_f<B, RW, SLOT>();     // most negative delta
};

template <int D>
__device__ __forceinline__ void red_imm(uint32_t a, int v) {
    asm volatile("red.shared.add.s32 [%0+%1], %2;" ::"r"(a), "n"(D), "r"(v) : "memory");
}
// a = byte address of the entry's site + 4 StMin (every immediate is >= 0)
template <int B, int RW, int SLOT, int... K>
__device__ __forceinline__ void fx_own(uint32_t a, const int (&w)[6], std::integer_sequence<int, K...>) {
    (red_imm<4 * (StOff<B, RW, SLOT, K>::delta - StMin<B, RW, SLOT>::v)>(a, w[StOff<B, RW, SLOT, K>::sh]), ...);
}
// halo-row entry: the term lands in the strip iff h + dyc < ty (h = halo row - 2, unsigned)
template <int B, int RW, int SLOT, int... K>
__device__ __forceinline__ void fx_halo(uint32_t a, const int (&w)[6], uint32_t h, uint32_t ty,
                                        std::integer_sequence<int, K...>) {
    ((h + (uint32_t)(int)StOff<B, RW, SLOT, K>::dyc < ty
          ? red_imm<4 * (StOff<B, RW, SLOT, K>::delta - StMin<B, RW, SLOT>::v)>(a, w[StOff<B, RW, SLOT, K>::sh])
          : void()),
     ...);
}

template <int LG, int TYG>
__device__ void strip_fast(const VoxelDev& V, const int4 it, int32_t* buf, uint32_t* lists,
                           const int (*cq8)[8], const int32_t* sph, int* cnt2, int32_t rho0) {
    constexpr int RW = 2 * LG + 2 * kRowPad, SLOT = (TYG + 2 * kGuard) * RW + 4;
    using Seq = std::make_integer_sequence<int, kSph>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = V.L, M2 = 2 * L, nq = M2 / 4;
    const int y0 = it.y, z0 = it.z, tz = it.w & 0xFFFF;
    const int ty = min(TYG, L - y0);
    const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(buf);
    for (int pr = warp; pr < kPlanes * (ty + 2 * kGuard); pr += kStripThreads / 32) {
        const int p = pr / (ty + 2 * kGuard), br = pr - p * (ty + 2 * kGuard);
        int32_t* row = buf + p * SLOT + br * RW;
        const bool own = br >= kGuard && br < ty + kGuard;
        for (int c = lane; c < RW; c += 32) row[c] = own && c >= kRowPad && c < kRowPad + M2 ? rho0 : 0;
    }
    auto wrap = [&](int z) { return z < 0 ? z + L : (z >= L ? z - L : z); };
    const int n_src = tz + 4;
    const int cpr = M2 / 16, per_plane = (ty + 4) * cpr;
    int ck_pl[kChunks], ck_hr[kChunks], ck_u[kChunks], ck_off[kChunks];
#pragma unroll
    for (int k = 0; k < kChunks; ++k) {
        const int c = tid + k * kStripThreads;
        const int pl = c / per_plane, rem = c - pl * per_plane;
        const int hr = rem / cpr, cx = rem - hr * cpr;
        ck_pl[k] = pl;
        ck_hr[k] = hr;
        ck_u[k] = (pl + 2) * SLOT + hr * RW + 16 * cx + kRowPad;
        ck_off[k] = wrap(y0 - 2 + hr) * M2 + 16 * cx;
    }
    uint4 v[kChunks];
    auto load_block = [&](int rb) {
        const int nb = min(kBlk, n_src - rb);
#pragma unroll
        for (int k = 0; k < kChunks; ++k)
            if (ck_pl[k] < nb)
                v[k] = __ldcs((const uint4*)(V.species + (size_t)wrap(z0 - 2 + rb + ck_pl[k]) * L * M2 + ck_off[k]));
    };
    // list building of the block at rb (its chunks are in v), into counters cnt
    auto append = [&](int rb, int* cnt) {
        const int nb = min(kBlk, n_src - rb);
#pragma unroll
        for (int k = 0; k < kChunks; ++k) {
            if (ck_pl[k] >= nb) break;
            uint32_t M = nonzero_bytes(v[k]);
            if (!M) continue;
            const int hr = ck_hr[k];
            const bool own = strip_own(hr, ty);
            const uint32_t M0 = M & 0x5555u, M1 = M & 0xAAAAu;
            int a0 = M0 ? atomicAdd(&cnt[own ? 0 : 1], __popc(M0)) : 0;
            int a1 = M1 ? atomicAdd(&cnt[own ? 2 : 3], __popc(M1)) : 0;
            while (M) {
                const int j = __ffs(M) - 1;
                M &= M - 1;
                const uint32_t wj = j < 8 ? (j < 4 ? v[k].x : v[k].y) : (j < 12 ? v[k].z : v[k].w);
                const uint32_t en = strip_entry((wj >> (8 * (j & 3))) & 0xFFu, ck_u[k] + j, hr);
                if (j & 1) strip_push(lists, en, 1, own, a1++);
                else strip_push(lists, en, 0, own, a0++);
            }
        }
    };
    if (tid < 8) cnt2[tid] = 0;
    load_block(0);
    __syncthreads();
    append(0, cnt2);
    if (kBlk < n_src) load_block(kBlk);
    __syncthreads();
    const int4 pure = make_int4(rho0, rho0, rho0, rho0);
    int qb = -2, par = 0;
    for (int rb = 0; rb < n_src; rb += kBlk, qb += kBlk, par ^= 1) {
        const int nb = min(kBlk, n_src - rb);
        int* cnt = cnt2 + 4 * par;
        // b. scatter of block rb; the counters of block rb + 4 are cleared meanwhile
        const int n0 = cnt[0], n1 = cnt[1], n2 = cnt[2], n3 = cnt[3];
        if (tid < 4) cnt2[4 * (par ^ 1) + tid] = 0;
        if (n0 + n1 <= kStripCap && n2 + n3 <= kStripCap) {
            const int c0 = (n0 + 31) >> 5, c1 = c0 + ((n1 + 31) >> 5), c2 = c1 + ((n2 + 31) >> 5),
                      c3 = c2 + ((n3 + 31) >> 5);
            for (int c = warp; c < c3; c += kStripThreads / 32) {
                const int lst = c < c0 ? 0 : c < c1 ? 1 : c < c2 ? 2 : 3;      // warp-uniform
                const int i = 32 * (c - (lst == 0 ? 0 : lst == 1 ? c0 : lst == 2 ? c1 : c2)) + lane;
                const int n = lst == 0 ? n0 : lst == 1 ? n1 : lst == 2 ? n2 : n3;
                if (i >= n) continue;
                const int b = lst >> 1;
                const uint32_t en = lists[b * kStripCap + ((lst & 1) ? kStripCap - 1 - i : i)];
                const int4 wa = *(const int4*)cq8[en & 7], wb = *(const int4*)(cq8[en & 7] + 4);
                const int w[6] = {0, wa.y, wa.z, wa.w, wb.x, wb.y};
                const uint32_t a = sbuf + 4 * ((en >> 3) & 0xFFFFFu);
                const uint32_t h = (en >> 23) - 2u;
                constexpr uint32_t m0 = 4u * (uint32_t)-StMin<0, RW, SLOT>::v, m1 = 4u * (uint32_t)-StMin<1, RW, SLOT>::v;
                if (lst == 0) fx_own<0, RW, SLOT>(a - m0, w, Seq{});
                else if (lst == 1) fx_halo<0, RW, SLOT>(a - m0, w, h, (uint32_t)ty, Seq{});
                else if (lst == 2) fx_own<1, RW, SLOT>(a - m1, w, Seq{});
                else fx_halo<1, RW, SLOT>(a - m1, w, h, (uint32_t)ty, Seq{});
            }
        } else {
            // direct scatter of the block, one source site per thread and pass
            const int nsite = nb * (ty + 4) * M2;
            for (int c = tid; c < nsite; c += kStripThreads) {
                const int pl = c / ((ty + 4) * M2), rem = c - pl * (ty + 4) * M2, hr = rem / M2, X = rem - hr * M2;
                uint32_t sp = V.species[((size_t)wrap(z0 - 2 + rb + pl) * L + wrap(y0 - 2 + hr)) * M2 + X];
                if (sp == 0) continue;
                sp = sp > 7 ? 7 : sp;
                const int bb = X & 1, u = (pl + 2) * SLOT + hr * RW + X + kRowPad;
                for (int k = 0; k < kSph; ++k) {
                    const int o = sph[k];
                    const int dyc = half_floor(bb + off_dy(o)), dzc = half_floor(bb + off_dz(o));
                    if ((unsigned)(hr + dyc - 2) < (unsigned)ty)
                        atomicAdd(buf + u + dzc * SLOT + dyc * RW + off_dx(o), cq8[sp][off_extra(o)]);
                }
            }
        }
        __syncthreads();
        // c. planes 0..3 are complete: row pads folded into the row ends, 16-byte
        // stores (planes outside the CTA's z range dropped); planes 4..7 move down
        // (pads included) and restart as pure Fe.  The next block's lists are built
        // in the same phase.
#pragma unroll 1
        for (int i = 0; i < kBlk; ++i) {
            const int q = qb + i;
            const bool wr = q >= 2 && q < tz + 2;
            int4* out = (int4*)(V.rho + ((size_t)(z0 + q - 2) * L + y0) * M2);
            for (int r = warp; r < ty; r += kStripThreads / 32) {
                int32_t* rowi = buf + i * SLOT + (r + kGuard) * RW + kRowPad;
                int32_t* upi = rowi + kBlk * SLOT;
                int4* row = (int4*)rowi;
                int4* up = (int4*)upi;
                int4* orow = out + r * nq;
                for (int c = lane; c < nq; c += 32) {
                    int4 val = row[c];
                    if (c == 0) {             // right pads (X = 2L .. 2L+2) into sites 0..2
                        val.x += rowi[M2];
                        val.y += rowi[M2 + 1];
                        val.z += rowi[M2 + 2];
                        row[nq] = up[nq];
                        up[nq] = make_int4(0, 0, 0, 0);
                    }
                    if (c == nq - 1) {        // left pads (X = -3 .. -1) into sites 2L-3 .. 2L-1
                        val.y += rowi[-3];
                        val.z += rowi[-2];
                        val.w += rowi[-1];
                        row[-1] = up[-1];
                        up[-1] = make_int4(0, 0, 0, 0);
                    }
                    if (wr) __stcs(orow + c, val);
                    row[c] = up[c];
                    up[c] = pure;
                }
            }
        }
        if (rb + kBlk < n_src) {
            append(rb + kBlk, cnt2 + 4 * (par ^ 1));
            if (rb + 2 * kBlk < n_src) load_block(rb + 2 * kBlk);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kStripThreads, 2) density_strip_kernel(const VoxelDev* vox, const ModelDev* M,
                                                                         const Tables* tab, const int4* items) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int4 s_wt[8][8][2];      // [species][sub]: f_s - f_Fe at the 8 offsets k = sub + 8j
    __shared__ __align__(16) int32_t s_cq8[8][8];   // [species][shell]: f_s - f_Fe (0 for Fe and codes > 4)
    __shared__ int32_t s_sph[64];
    __shared__ int s_count[8];
    const int4 it = items[blockIdx.x];
    const int tid = threadIdx.x;
    if (tid < kSph) s_sph[tid] = tab->sph_off[tid];
    if (tid < 64) s_cq8[tid >> 3][tid & 7] = (tid >> 3) >= 1 && (tid >> 3) <= 4 ? M->cq[tid >> 3][tid & 7] : 0;
    __syncthreads();
    const VoxelDev& V = vox[it.x];
    const int L = V.L;
    int32_t* buf = (int32_t*)sm;
    if (((it.w >> 16) & 1) && L <= 128) {
        const int LG = strip_geom_L(L);
        uint32_t* lists = (uint32_t*)(sm + sizeof(int32_t) * (size_t)kPlanes * strip_slot(strip_rows(L), LG));
        if (LG == 32)
            strip_fast<32, 16>(V, it, buf, lists, s_cq8, s_sph, s_count, M->rho_pure);
        else if (LG == 64)
            strip_fast<64, 16>(V, it, buf, lists, s_cq8, s_sph, s_count, M->rho_pure);
        else
            strip_fast<128, 8>(V, it, buf, lists, s_cq8, s_sph, s_count, M->rho_pure);
        return;
    }
    for (int i = tid; i < 8 * 8 * 8; i += kStripThreads) {
        const int sp = i >> 6, sub = (i >> 3) & 7, j = i & 7, k = sub + 8 * j;
        ((int32_t*)s_wt)[i] = (sp >= 1 && sp <= 4 && k < kSph) ? M->cq[sp][off_extra(s_sph[k])] : 0;
    }
    __syncthreads();
    const int TY = it.w >> 17;
    uint32_t* lists = (uint32_t*)(sm + sizeof(int32_t) * (size_t)kPlanes * strip_slot(TY, L));
    if ((it.w >> 16) & 1)
        strip_body<true>(V, it, buf, lists, s_wt, s_sph, s_count, M->rho_pure);
    else
        strip_body<false>(V, it, buf, lists, s_wt, s_sph, s_count, M->rho_pure);
}

int density_strip_rows(int L) { return strip_rows(L); }
// a 16-byte strip of L <= 128 takes the fixed geometry of strip_geom_L(L), which
// holds the byte path's layout too
size_t density_strip_smem(int L) { return strip_smem(strip_rows(L), L <= 128 ? strip_geom_L(L) : L); }

cudaError_t launch_density(const VoxelDev* vox, const ModelDev* M, const Tables* tab, const int4* tiles,
                           int n_tiles, const int4* strips, int n_strips, size_t strip_dyn, cudaStream_t st) {
    if (n_strips > 0) {
        cudaError_t e = cudaFuncSetAttribute((const void*)density_strip_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)strip_dyn);
        if (e != cudaSuccess) return e;
        density_strip_kernel<<<n_strips, kStripThreads, strip_dyn, st>>>(vox, M, tab, strips);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_tiles > 0) {
        const size_t dyn = sizeof(int32_t) * kTX * kTY * kTZ * 2 +
                           (size_t)(kTX + 2 * kHalo) * (kTY + 2 * kHalo) * (kTZ + 2 * kHalo) * 2;
        cudaError_t e = cudaFuncSetAttribute((const void*)density_tile_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        density_tile_kernel<<<n_tiles, kDensThreads, dyn, st>>>(vox, M, tab, tiles);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace akmc
