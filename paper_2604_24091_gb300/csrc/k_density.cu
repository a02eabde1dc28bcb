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
// voxel.  It walks the source planes z0-2 .. z0+tz+1 once, in order: each
// plane's haloed strip of species rows (ty+4 rows of 2L sites, one 16-byte
// vector load per thread, prefetched one plane ahead) is scanned for non-Fe
// sites, which are appended to a list (warp scan, one shared atomic per
// warp); then 8 lanes per listed site add its 58 corrections f_s - f_Fe to a
// buffer of 8 density planes in shared memory (each lane 7 or 8 offsets, the
// offsets' buffer deltas held in registers).  The buffer holds planes
// [qb, qb+8); after the 4 source planes qb+2 .. qb+5 the planes qb .. qb+3 are
// complete: they are written to memory with 16-byte stores (planes outside
// the CTA's range are dropped), planes qb+4 .. qb+7 move down and the top
// half restarts as pure Fe.  Rows are padded by 4 sites on each side, so an x
// offset needs no wrap: the pads are folded into the row ends when a plane is
// written.
//
// Site coordinates: within a row (fixed y, z) the site index 2x+b equals the
// half-unit coordinate X, so a neighbour at half-unit offset dx sits at
// X + dx (mod 2L) of the row that holds cell floor((Y + dy)/2).
//
// Per output site the work is one species byte read, one density write and,
// for the ~2% non-Fe sites (x the halo factor (ty+4)/ty * (tz+4)/tz), 58
// shared-memory atomics.

constexpr int kStripThreads = 256;
constexpr int kStripWarps = kStripThreads / 32;
constexpr int kPlanes = 8;          // density planes held
constexpr int kShift = 4;           // planes completed per block of source planes
constexpr int kRowPad = 4;          // padding sites on each side of a buffer row
constexpr int kLanesPerSite = 8;    // scatter lanes per listed site

__host__ __device__ inline int strip_rw(int L) { return 2 * L + 2 * kRowPad; }
__host__ __device__ inline int strip_slot(int TY, int L) { return TY * strip_rw(L) + 4; }

// floor((b + d) / 2) for b in {0,1}, d in [-4, 4]
__device__ __forceinline__ int half_floor(int v) { return (v + 8) / 2 - 4; }

// Entries of rows hr in [4, ty) reach only rows inside the strip and go to the
// front of the list (count[0]); the others go to the back (count[1], list
// index cap - 1 - i) and are scattered with a row check.
__device__ __forceinline__ bool strip_inner(int hr, int ty) { return hr >= 4 && hr < ty; }

template <bool VEC>
__device__ __forceinline__ void strip_append(const uint8_t* sp, int L, int zp, int y0, int ty, uint4 pre,
                                             int my_hr, int my_cx, uint32_t* list, int cap, int* count) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int M2 = 2 * L;
    if (VEC) {
        // the chunk this thread loaded: 16 sites X = 16 cx .. 16 cx + 15 of halo row hr
        uint32_t M = 0;
        if (my_hr >= 0) {
            const uint32_t w[4] = {pre.x, pre.y, pre.z, pre.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t t = w[i] | (w[i] >> 4);
                t |= t >> 2;
                t |= t >> 1;
                t &= 0x01010101u;                       // bit 0 of each byte: byte != 0
                M |= ((t | (t >> 7) | (t >> 14) | (t >> 21)) & 0xFu) << (4 * i);
            }
        }
        if (M) {
            const int c = __popc(M);
            const bool in = strip_inner(my_hr, ty);
            const int at0 = atomicAdd(&count[in ? 0 : 1], c);
            int i = 0;
            while (M) {
                const int j = __ffs(M) - 1;
                M &= M - 1;
                const uint32_t wj = j < 8 ? (j < 4 ? pre.x : pre.y) : (j < 12 ? pre.z : pre.w);
                const uint32_t s = (wj >> (8 * (j & 3))) & 0xFFu;
                const uint32_t en = (s > 7 ? 7u : s) | ((uint32_t)(16 * my_cx + j) << 3) | ((uint32_t)my_hr << 13);
                list[in ? at0 + i : cap - 1 - (at0 + i)] = en;
                ++i;
            }
        }
        (void)lane;
    } else {
        // byte path (rows not 16-byte aligned): one byte per thread and pass
        const int n = (ty + 4) * M2;
        for (int c0 = 0; c0 < n; c0 += kStripThreads) {
            const int c = c0 + tid;
            uint32_t s = 0;
            int hr = 0, X = 0;
            if (c < n) {
                hr = c / M2;
                X = c - hr * M2;
                int y = y0 - 2 + hr;
                y = y < 0 ? y + L : (y >= L ? y - L : y);
                s = sp[((size_t)zp * L + y) * M2 + X];
            }
            const bool hit = s != 0, in = strip_inner(hr, ty);
            const unsigned mi = __ballot_sync(0xffffffffu, hit && in), me = __ballot_sync(0xffffffffu, hit && !in);
            int bi = 0, be = 0;
            if (lane == 0 && mi) bi = atomicAdd(&count[0], __popc(mi));
            if (lane == 0 && me) be = atomicAdd(&count[1], __popc(me));
            bi = __shfl_sync(0xffffffffu, bi, 0);
            be = __shfl_sync(0xffffffffu, be, 0);
            const uint32_t en = (s > 7 ? 7u : s) | ((uint32_t)X << 3) | ((uint32_t)hr << 13);
            if (hit && in) list[bi + __popc(mi & ((1u << lane) - 1u))] = en;
            if (hit && !in) list[cap - 1 - (be + __popc(me & ((1u << lane) - 1u)))] = en;
        }
    }
}

// Planes buf[0..3] are complete: write those inside the CTA's range (rel. plane
// q in [2, tz+2), i.e. z = z0 + q - 2), move buf[4..7] down, reset buf[4..7].
// Every element is read, moved and reset by the same thread.
template <bool VEC>
__device__ void strip_shift(const VoxelDev& V, int32_t* buf, int SLOT, int RW, int ty, int y0, int z0, int qb,
                            int tz, int32_t rho0) {
    const int L = V.L, M2 = 2 * L;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (VEC) {
        const int C = RW / 4;                     // int4 per padded row (RW = 2L + 8, L even)
        const int c_first = kRowPad / 4, c_last = (kRowPad + M2) / 4 - 1;
        const int4 pure = make_int4(rho0, rho0, rho0, rho0), zero = make_int4(0, 0, 0, 0);
        for (int r = warp; r < ty; r += kStripWarps) {
            for (int c = lane; c < C; c += 32) {
                if (c < c_first || c > c_last) continue;
#pragma unroll
                for (int i = 0; i < kShift; ++i) {
                    const int32_t* row = buf + i * SLOT + r * RW;
                    const int q = qb + i;
                    if (q < 2 || q >= tz + 2) continue;
                    int4 v = *(const int4*)(row + 4 * c);
                    if (c == c_first) {            // sites 0..2 collect the right pads (X = 2L .. 2L+2)
                        v.x += row[kRowPad + M2];
                        v.y += row[kRowPad + M2 + 1];
                        v.z += row[kRowPad + M2 + 2];
                    }
                    if (c == c_last) {             // sites 2L-3..2L-1 collect the left pads (X = -3 .. -1)
                        v.y += row[kRowPad - 3];
                        v.z += row[kRowPad - 2];
                        v.w += row[kRowPad - 1];
                    }
                    *(int4*)(V.rho + ((size_t)(z0 + q - 2) * L + y0 + r) * M2 + 4 * (c - c_first)) = v;
                }
            }
            __syncwarp();   // every read of this row (pads included) precedes the moves below
            for (int c = lane; c < C; c += 32) {
                const bool site = c >= c_first && c <= c_last;
#pragma unroll
                for (int i = 0; i < kShift; ++i) {
                    int32_t* row = buf + i * SLOT + r * RW;
                    int32_t* up = buf + (i + kShift) * SLOT + r * RW;
                    *(int4*)(row + 4 * c) = *(const int4*)(up + 4 * c);
                    *(int4*)(up + 4 * c) = site ? pure : zero;
                }
            }
        }
    } else {
        for (int r = warp; r < ty; r += kStripWarps) {
            for (int i = 0; i < kShift; ++i) {
                int32_t* row = buf + i * SLOT + r * RW + kRowPad;
                const int q = qb + i;
                if (q >= 2 && q < tz + 2) {
                    int32_t* out = V.rho + ((size_t)(z0 + q - 2) * L + y0 + r) * M2;
                    for (int c = lane; c < M2; c += 32) {
                        int v = row[c];
                        if (c < 3) v += row[M2 + c];
                        if (c >= M2 - 3) v += row[c - M2];
                        out[c] = v;
                    }
                }
            }
            __syncwarp();
            for (int i = 0; i < kShift; ++i) {
                int32_t* row = buf + i * SLOT + r * RW;
                int32_t* up = buf + (i + kShift) * SLOT + r * RW;
                for (int c = lane; c < RW; c += 32) {
                    row[c] = up[c];
                    up[c] = (c >= kRowPad && c < kRowPad + M2) ? rho0 : 0;
                }
            }
        }
    }
}

template <bool VEC>
__device__ void strip_body(const VoxelDev& V, const int4 it, int TY, int32_t* buf, uint32_t* lists, int list_cap,
                           const int32_t (*cq)[8], const int32_t* sph, int* counts, int32_t rho0) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = V.L, M2 = 2 * L;
    const int y0 = it.y, z0 = it.z, tz = it.w & 0xFFFF;
    const int ty = min(TY, L - y0);
    const int RW = strip_rw(L), SLOT = strip_slot(TY, L);
    // this lane's stencil offsets k = sub + 8j: buffer delta dzc*SLOT + dyc*RW + dx
    // (15 bits, biased), dyc + 2 (3 bits), shell (3 bits); one word per b
    const int sub = tid & (kLanesPerSite - 1);
    uint32_t P0[8], P1[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = sub + kLanesPerSite * j;
        const int o = k < kSph ? sph[k] : sph[0];
        const int dx = off_dx(o), dy = off_dy(o), dz = off_dz(o);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int dyc = half_floor(b + dy), dzc = half_floor(b + dz);
            const uint32_t w = (uint32_t)(dzc * SLOT + dyc * RW + dx + 16384) | ((uint32_t)(dyc + 2) << 15) |
                               ((uint32_t)off_extra(o) << 18);
            if (b) P1[j] = w; else P0[j] = w;
        }
    }
    // buffer: planes qb .. qb+7 (relative plane index; rel. plane 2 is z0), all pure Fe
    for (int r = warp; r < kPlanes * ty; r += kStripWarps) {
        int32_t* row = buf + (r / ty) * SLOT + (r % ty) * RW;
        for (int c = lane; c < RW; c += 32) row[c] = (c >= kRowPad && c < kRowPad + M2) ? rho0 : 0;
    }
    // this thread's chunk of the haloed strip (VEC: 16 sites of one row)
    int my_hr = -1, my_cx = 0, my_y = -1;
    if (VEC) {
        const int cpr = M2 / 16;
        if (tid < (ty + 4) * cpr) {
            my_hr = tid / cpr;
            my_cx = tid - my_hr * cpr;
            int y = y0 - 2 + my_hr;
            my_y = y < 0 ? y + L : (y >= L ? y - L : y);
        }
    }
    auto plane_of = [&](int rp) { int z = z0 - 2 + rp; return z < 0 ? z + L : (z >= L ? z - L : z); };
    auto load = [&](int rp, uint4& v) {
        if (VEC && my_y >= 0) v = *(const uint4*)(V.species + ((size_t)plane_of(rp) * L + my_y) * M2 + 16 * my_cx);
    };
    uint4 pre = make_uint4(0, 0, 0, 0);
    load(0, pre);
    if (tid < 4) counts[tid] = 0;
    __syncthreads();
    const int n_src = tz + 4;
    int qb = -2;
    for (int rp = 0; rp < n_src; ++rp) {
        const uint4 cur = pre;
        if (rp + 1 < n_src) load(rp + 1, pre);
        uint32_t* list = lists + (rp & 1) * list_cap;
        int* cnt = counts + 2 * (rp & 1);
        strip_append<VEC>(V.species, L, plane_of(rp), y0, ty, cur, my_hr, my_cx, list, list_cap, cnt);
        __syncthreads();
        const int pos = rp - qb;                      // 2 .. 5: targets at buffer planes pos-2 .. pos+2
        // entries of inner rows: every target row lies in the strip
        const int ni = cnt[0] * kLanesPerSite;
        for (int t = tid; t < ni; t += kStripThreads) {
            const uint32_t en = list[t / kLanesPerSite];
            const int s = en & 7, X = (en >> 3) & 1023, hr = en >> 13;
            const int u = pos * SLOT + (hr - 2) * RW + X + kRowPad - 16384;
            const int32_t* cs = cq[s];
            const bool b = X & 1;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j == 7 && sub + kLanesPerSite * j >= kSph) break;
                const uint32_t w = b ? P1[j] : P0[j];
                atomicAdd(buf + (u + (int)(w & 0x7FFF)), cs[w >> 18]);
            }
        }
        // entries of edge rows: row check
        const int ne = cnt[1] * kLanesPerSite;
        for (int t = tid; t < ne; t += kStripThreads) {
            const uint32_t en = list[list_cap - 1 - t / kLanesPerSite];
            const int s = en & 7, X = (en >> 3) & 1023, hr = en >> 13;
            const int u = pos * SLOT + (hr - 2) * RW + X + kRowPad - 16384;
            const int hm = hr - 4;                    // target row hr + dyc - 2 = hm + (dyc + 2)
            const int32_t* cs = cq[s];
            const bool b = X & 1;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j == 7 && sub + kLanesPerSite * j >= kSph) break;
                const uint32_t w = b ? P1[j] : P0[j];
                if ((unsigned)(hm + (int)((w >> 15) & 7)) < (unsigned)ty)
                    atomicAdd(buf + (u + (int)(w & 0x7FFF)), cs[w >> 18]);
            }
        }
        if (tid < 2) counts[2 * ((rp + 1) & 1) + tid] = 0;
        __syncthreads();
        if (pos == kShift + 1) {                      // buffer planes 0..3 complete
            strip_shift<VEC>(V, buf, SLOT, RW, ty, y0, z0, qb, tz, rho0);
            qb += kShift;
        }
    }
    // flush: every source plane is done; the planes still to be written (at
    // most 3: the last shift came after source plane tz or later) sit in
    // buffer planes 0..3
    strip_shift<VEC>(V, buf, SLOT, RW, ty, y0, z0, qb, tz, rho0);
}

__global__ void __launch_bounds__(kStripThreads) density_strip_kernel(const VoxelDev* vox, const ModelDev* M,
                                                                      const Tables* tab, const int4* items, int TY,
                                                                      int buf_ints, int list_cap) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int32_t s_cq[8][8];
    __shared__ int32_t s_sph[64];
    __shared__ int s_count[4];
    const int4 it = items[blockIdx.x];
    const int tid = threadIdx.x;
    if (tid < kSph) s_sph[tid] = tab->sph_off[tid];
    if (tid < 64) s_cq[tid / 8][tid % 8] = tid < 40 ? M->cq[tid / 8][tid % 8] : 0;
    __syncthreads();
    int32_t* buf = (int32_t*)sm;
    uint32_t* lists = (uint32_t*)(sm + sizeof(int32_t) * (size_t)buf_ints);
    const VoxelDev& V = vox[it.x];
    if (it.w >> 16)
        strip_body<true>(V, it, TY, buf, lists, list_cap, s_cq, s_sph, s_count, M->rho_pure);
    else
        strip_body<false>(V, it, TY, buf, lists, list_cap, s_cq, s_sph, s_count, M->rho_pure);
}

cudaError_t launch_density(const VoxelDev* vox, const ModelDev* M, const Tables* tab, const int4* tiles,
                           int n_tiles, const int4* strips, int n_strips, int strip_ty, int strip_lmax,
                           cudaStream_t st) {
    if (n_strips > 0) {
        const int buf_ints = kPlanes * strip_slot(strip_ty, strip_lmax);
        const int list_cap = (strip_ty + 4) * 2 * strip_lmax;
        const size_t dyn = sizeof(int32_t) * (size_t)buf_ints + 2 * sizeof(uint32_t) * (size_t)list_cap;
        cudaError_t e = cudaFuncSetAttribute((const void*)density_strip_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        density_strip_kernel<<<n_strips, kStripThreads, dyn, st>>>(vox, M, tab, strips, strip_ty, buf_ints,
                                                                   list_cap);
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
