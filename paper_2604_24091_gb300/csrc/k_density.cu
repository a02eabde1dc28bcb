// k_density.cu -- EAM site densities from the lattice (build_density):
//   rho_i = sum_{j in S(i), s_j != V} f_{s_j}(r_ij)   (fixed point, exact).
//
// Streaming stencil over tiles of 32 x 16 x 16 cells.  A perfect-Fe lattice
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

__global__ void __launch_bounds__(kDensThreads) density_kernel(const VoxelDev* vox, const ModelDev* M,
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

cudaError_t launch_density(const VoxelDev* vox, const ModelDev* M, const Tables* tab,
                           const int4* items, int n_items, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const size_t dyn = sizeof(int32_t) * kTX * kTY * kTZ * 2 +
                       (size_t)(kTX + 2 * kHalo) * (kTY + 2 * kHalo) * (kTZ + 2 * kHalo) * 2;
    cudaError_t e = cudaFuncSetAttribute((const void*)density_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    density_kernel<<<n_items, kDensThreads, dyn, st>>>(vox, M, tab, items);
    return cudaGetLastError();
}

}  // namespace akmc
