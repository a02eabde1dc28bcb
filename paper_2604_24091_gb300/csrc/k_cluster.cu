// k_cluster.cu -- Cu cluster size histogram of one voxel (observable).
// Clusters are connected components of Cu sites under 1nn+2nn (mode 0) or
// 1nn (mode 1) adjacency.  Lock-free union-find over site labels: every
// parent pointer points to a smaller site index, links go from the larger
// root to the smaller one with compare-and-swap, so every loop below ends
// after at most N iterations.  Scratch: labels[N], sizes[N] (int32).
#include <akmc.h>

#include <mutex>
#include <string>

#include "akmc_device.cuh"
#include "akmc_launch.h"

namespace akmc {

__device__ __forceinline__ int uf_find(int32_t* lab, int x) {
    int p = lab[x];
    while (p != x) {
        int gp = lab[p];
        if (gp != p) lab[x] = gp;   // path halving; gp is still an ancestor of x
        x = p;
        p = gp;
    }
    return x;
}

__device__ __forceinline__ void uf_union(int32_t* lab, int a, int b) {
    for (;;) {
        a = uf_find(lab, a);
        b = uf_find(lab, b);
        if (a == b) return;
        if (a > b) { int t = a; a = b; b = t; }
        int old = atomicCAS(&lab[b], b, a);
        if (old == b) return;
        b = old;
    }
}

__global__ void cluster_init(const uint8_t* sp, int N, int32_t* lab, int32_t* sizes) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        lab[i] = sp[i] == 1 ? i : -1;
        sizes[i] = 0;
    }
}

__global__ void cluster_hook(const uint8_t* sp, int L, int N, const Tables* tab, int n_adj, int32_t* lab) {
    const int M2 = 2 * L;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        if (sp[i] != 1) continue;
        const int b = i & 1, c = i >> 1;
        const int X = 2 * (c % L) + b, Y = 2 * ((c / L) % L) + b, Z = 2 * (c / (L * L)) + b;
        for (int k = 0; k < n_adj; ++k) {
            const int o = tab->sph_off[k];
            const int j = site_index(wrap_coord(X + off_dx(o), M2), wrap_coord(Y + off_dy(o), M2),
                                     wrap_coord(Z + off_dz(o), M2), L);
            if (j > i && sp[j] == 1) uf_union(lab, i, j);
        }
    }
}

__global__ void cluster_count(int N, int32_t* lab, int32_t* sizes) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        if (lab[i] < 0) continue;
        atomicAdd(&sizes[uf_find(lab, i)], 1);
    }
}

__global__ void cluster_bins(int N, const int32_t* lab, const int32_t* sizes, unsigned long long* hist) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        if (lab[i] != i) continue;
        const int s = sizes[i];
        const int bin = s <= 4 ? s - 1 : (s < 10 ? 4 : (s < 20 ? 5 : (s < 50 ? 6 : 7)));
        atomicAdd(&hist[bin], 1ull);
    }
}

static cudaError_t launch_cluster_raw(const uint8_t* species, int L, int N, const Tables* tab, int mode,
                                      int32_t* labels, int32_t* sizes, unsigned long long* hist, cudaStream_t st) {
    const int threads = 256;
    int blocks = (N + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    cudaError_t e = cudaMemsetAsync(hist, 0, 8 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    cluster_init<<<blocks, threads, 0, st>>>(species, N, labels, sizes);
    cluster_hook<<<blocks, threads, 0, st>>>(species, L, N, tab, mode == 0 ? 14 : 8, labels);
    cluster_count<<<blocks, threads, 0, st>>>(N, labels, sizes);
    cluster_bins<<<blocks, threads, 0, st>>>(N, labels, sizes, hist);
    return cudaGetLastError();
}

cudaError_t launch_cluster(const VoxelDev* vox_host, int voxel, int N, const Tables* tab, int mode,
                           int32_t* labels, int32_t* sizes, unsigned long long* hist, cudaStream_t st) {
    const VoxelDev& V = vox_host[voxel];
    return launch_cluster_raw(V.species, V.L, N, tab, mode, labels, sizes, hist, st);
}

}  // namespace akmc

// ---- allocation-free entry point ---------------------------------------------
// Some callers cannot let a library allocate device memory: programs whose
// GPU memory is owned entirely by another allocator (a framework or
// simulation that reserves the device's memory up front and treats any other
// cudaMalloc as an error or a source of fragmentation), and code on a
// latency-critical path where an allocation may block or synchronise the
// device.  For them the Cu cluster histogram has a variant whose scratch
// (union-find labels and cluster sizes) is a fixed file-scope device array;
// the caller passes only its input lattice and its output histogram.

namespace {

constexpr int kStaticMaxSites = 2 * 64 * 64 * 64;   // 524,288 sites: lattices up to L = 64
static __device__ __align__(256) int32_t g_cluster_scratch[2 * kStaticMaxSites];
static __device__ __align__(256) akmc::Tables g_static_tables;

struct StaticSetup {
    bool done = false;
    int32_t* scratch = nullptr;
    akmc::Tables* tables = nullptr;
};
std::mutex g_static_mu;
StaticSetup g_static_setup[64];

akmc_status static_fail(akmc_status st, const std::string& msg) {
    akmc::set_last_error(msg.c_str());
    return st;
}

}  // namespace

extern "C" akmc_status akmc_cluster_hist_noalloc(const uint8_t* species, int32_t L, int32_t mode, int64_t* hist,
                                                 akmc_stream stream) {
    using namespace akmc;
    if (!species || !hist) return static_fail(AKMC_EINVAL, "species or hist is NULL");
    if (mode != 0 && mode != 1) return static_fail(AKMC_EINVAL, "mode must be 0 or 1");
    if (L < 3 || 2LL * L * L * L > kStaticMaxSites)
        return static_fail(AKMC_EINVAL, "L=" + std::to_string(L) + " outside [3, 64]: the static scratch holds " +
                                             std::to_string(kStaticMaxSites) + " sites");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(AKMC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return static_fail(AKMC_EINVAL, "device ordinal above 63");
    StaticSetup su;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        StaticSetup& s = g_static_setup[dev];
        if (!s.done) {
            // once per device, with that device current: device addresses of the
            // static arrays, and the stencil tables copied into place
            e = cudaGetSymbolAddress((void**)&s.scratch, g_cluster_scratch);
            if (e != cudaSuccess)
                return static_fail(AKMC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            e = cudaGetSymbolAddress((void**)&s.tables, g_static_tables);
            if (e != cudaSuccess)
                return static_fail(AKMC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            // A copy from pageable host memory may return before the data reach
            // the device; the kernels run on the caller's stream, which may be a
            // non-blocking one that nothing orders after this copy, so wait for it.
            e = cudaMemcpyToSymbol(g_static_tables, &host_tables(), sizeof(Tables));
            if (e != cudaSuccess)
                return static_fail(AKMC_ECUDA, std::string("cudaMemcpyToSymbol: ") + cudaGetErrorString(e));
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess)
                return static_fail(AKMC_ECUDA, std::string("cudaDeviceSynchronize: ") + cudaGetErrorString(e));
            s.done = true;
        }
        su = s;
    }
    const int N = 2 * L * L * L;
    e = launch_cluster_raw(species, L, N, su.tables, mode, su.scratch, su.scratch + kStaticMaxSites,
                           (unsigned long long*)hist, (cudaStream_t)stream);
    if (e != cudaSuccess) return static_fail(AKMC_ECUDA, std::string("cluster kernels: ") + cudaGetErrorString(e));
    return AKMC_OK;
}
