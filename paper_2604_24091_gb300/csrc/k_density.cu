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
// tile; index arithmetic is per row, not per site.
#include "akmc_device.cuh"
#include "akmc_launch.h"

namespace akmc {

constexpr int kDensThreads = 256;
constexpr int kDensWarps = kDensThreads / 32;

__global__ void __launch_bounds__(kDensThreads) density_kernel(const VoxelDev* vox, const ModelDev* M,
                                                               const Tables* tab, const int4* items) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int32_t s_off[64];
    __shared__ int32_t s_cq[5][8];
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
    // scatter corrections of every non-Fe site of the haloed tile
    for (int r = warp; r < hz * hy; r += kDensWarps) {
        const int cy = r % hy, cz = r / hy;
        const uint8_t* src = hs + r * hrow;
        for (int c = lane; c < hrow; c += 32) {
            const int s = src[c];
            if (s == kFe) continue;
            const int b = c & 1;
            const int HX = c, HY = 2 * cy + b, HZ = 2 * cz + b;   // half-unit coordinates in the halo frame
            for (int k = 0; k < kSph; ++k) {
                const int o = s_off[k];
                const int X = HX + off_dx(o), Y = HY + off_dy(o), Z = HZ + off_dz(o);
                if (X < 0 || Y < 0 || Z < 0) continue;
                const int ix = (X >> 1) - kHalo, iy = (Y >> 1) - kHalo, iz = (Z >> 1) - kHalo;
                if (ix < 0 || iy < 0 || iz < 0 || ix >= tx || iy >= ty || iz >= tz) continue;
                atomicAdd(&rt[(iz * ty + iy) * trow + 2 * ix + (X & 1)], s_cq[s][off_extra(o)]);
            }
        }
    }
    __syncthreads();
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
