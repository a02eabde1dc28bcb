// k_setup.cu -- model setup (shell constants, embedding coefficient tables)
// and seeded species placement (step a1).
#include "akmc_device.cuh"
#include "akmc_launch.h"

namespace akmc {

// Cubic Hermite on a uniform grid, evaluated with explicitly rounded float64
// operations in a fixed order (no fused multiply-add), so that shell
// constants come out identical on every machine that evaluates the same form.
__device__ double hermite_rn(const double* tab, int k, double t, double h) {
    double v0 = tab[2 * k], d0 = __dmul_rn(tab[2 * k + 1], h);
    double v1 = tab[2 * k + 2], d1 = __dmul_rn(tab[2 * k + 3], h);
    double t2 = __dmul_rn(t, t), t3 = __dmul_rn(t2, t);
    double h00 = __dadd_rn(__dsub_rn(__dmul_rn(2.0, t3), __dmul_rn(3.0, t2)), 1.0);
    double h10 = __dadd_rn(__dsub_rn(t3, __dmul_rn(2.0, t2)), t);
    double h01 = __dadd_rn(__dmul_rn(-2.0, t3), __dmul_rn(3.0, t2));
    double h11 = __dsub_rn(t3, t2);
    double s = __dadd_rn(__dmul_rn(h00, v0), __dmul_rn(h10, d0));
    s = __dadd_rn(s, __dmul_rn(h01, v1));
    return __dadd_rn(s, __dmul_rn(h11, d1));
}

__device__ double table_at_r(const double* tab, int n, double r_cut, double r) {
    double dr = __ddiv_rn(r_cut, (double)(n - 1));
    double x = __ddiv_rn(r, dr);
    int k = (int)floor(x);
    k = k > n - 2 ? n - 2 : (k < 0 ? 0 : k);
    return hermite_rn(tab, k, __dsub_rn(x, (double)k), dr);
}

// Shell constants of the rigid bcc lattice: phi_ab and f_b at the 5 shell
// radii r_s = (a/2) sqrt(3, 4, 8, 11, 12), f rounded to the 2^-24 density grid;
// then the embedding tables: per interval the Hermite cubic in Horner form
// F(t) = F_k + t (c1 + t (c2 + t c3)), t in [0,1), in FP64 and FP32, and the
// knot values in 2^-40 eV fixed point.
__global__ void setup_model_kernel(ModelDev* M, int32_t* batch_status) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    if (M->has_eam) {
        const int len2[6] = {0, 3, 4, 8, 11, 12};
        if (blockIdx.x == 0) {
            for (int i = threadIdx.x; i < 10 * 8; i += blockDim.x) {
                M->phi_d[i / 8][i % 8] = 0.0;
                M->phi_q[i / 8][i % 8] = 0;
            }
            for (int i = threadIdx.x; i < 5 * 8; i += blockDim.x) M->fq[i / 8][i % 8] = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < 14 * 5; i += blockDim.x) {
                int fn = i / 5, s = i % 5 + 1;
                double r = __dmul_rn(__dmul_rn(M->a, 0.5), __dsqrt_rn((double)len2[s]));
                if (fn < 10) {
                    double v = table_at_r(M->phi_tab + (size_t)fn * M->n_r * 2, M->n_r, M->r_cut, r);
                    M->phi_d[fn][s] = v;
                    M->phi_q[fn][s] = llround(v * 0x1p40);
                } else {
                    int b = fn - 10;
                    double v = table_at_r(M->f_tab + (size_t)b * M->n_r * 2, M->n_r, M->r_cut, r);
                    long long q = llround(v * 0x1p24);
                    if (q < 0 || q > (1 << 26)) atomicExch(batch_status, kEINVAL);
                    M->fq[b][s] = (int32_t)q;
                }
            }
            __syncthreads();
            if (threadIdx.x < 5 * 8) {
                int b = threadIdx.x / 8, s = threadIdx.x % 8;
                M->cq[b][s] = M->fq[b][s] - M->fq[kFe][s];
            }
            if (threadIdx.x == 0) {
                const int cnt[6] = {0, 8, 6, 12, 24, 8};
                long long pure = 0, mx = 0;
                for (int s = 1; s <= 5; ++s) {
                    pure += (long long)cnt[s] * M->fq[kFe][s];
                    int best = 0;
                    for (int b = 0; b < 4; ++b) best = max(best, M->fq[b][s]);
                    mx += (long long)cnt[s] * best;
                }
                if (mx >= (1LL << 30)) atomicExch(batch_status, kEINVAL);
                M->rho_pure = (int32_t)pure;
                M->rho_max = (int32_t)min(mx, (long long)(1 << 30));
            }
        }
        const int nint = M->n_rho - 1;
        const double h = M->rho_h;
        for (int i = tid; i < 4 * M->n_rho; i += nth) {
            int a = i / M->n_rho, k = i % M->n_rho;
            const double* T = M->F_tab + (size_t)a * M->n_rho * 2;
            double F0 = T[2 * k];
            M->Fq[i] = llround(F0 * 0x1p40);
            if (k < nint) {
                double d0 = T[2 * k + 1] * h, F1 = T[2 * k + 2], d1 = T[2 * k + 3] * h;
                double c1 = d0;
                double c2 = 3.0 * (F1 - F0) - (2.0 * d0 + d1);
                double c3 = 2.0 * (F0 - F1) + (d0 + d1);
                M->Fd[(size_t)a * nint + k] = Cubic64{F0, c1, c2, c3};
                M->Ff[i] = make_float4((float)c1, (float)c2, (float)c3, 0.f);
            } else {
                M->Ff[i] = make_float4(0.f, 0.f, 0.f, 0.f);   // the last knot itself: F = Fq exactly
            }
        }
    }
}

// (a1) Placement: species counts n_s = floor(frac_s N + 0.5); draw k of the
// placement stream gives site floor(r * N / 2^64) from 64 Philox bits; the
// draw is taken if the site still holds Fe.  Order: vacancies (slot = order
// of placement), Cu, Ni, Mn.  One warp per voxel evaluates 32 consecutive
// draws at once and resolves them in draw order (a draw is taken iff its site
// is Fe and no earlier draw of the same batch hit that site).
__global__ void place_kernel(VoxelDev* vox, int n_vox, const int32_t* list) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n_vox) return;
    VoxelDev& V = vox[list ? list[w] : w];
    const int N = V.N;
    int cnt[4];
    cnt[0] = V.nv;
    long long total = V.nv;
    for (int s = 0; s < 3; ++s) {
        cnt[s + 1] = (int)floor(V.frac[s] * (double)N + 0.5);
        total += cnt[s + 1];
    }
    if (lane == 0) for (int s = 0; s < 4; ++s) V.counts[s] = cnt[s];
    const uint32_t k0 = (uint32_t)V.seed, k1 = (uint32_t)(V.seed >> 32);
    const uint32_t w2 = (uint32_t)V.uid, w3 = 0x80000000u | (uint32_t)(V.uid >> 32);
    const uint64_t max_draws = 64ull * (uint64_t)N + 65536ull;
    uint8_t* sp = V.species;
    long long placed = 0;
    uint64_t kb = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    while (placed < total) {
        if (kb > max_draws) {
            if (lane == 0) V.status = kEINVAL;
            return;
        }
        uint64_t k = kb + lane;
        uint32_t c0 = (uint32_t)k, c1 = (uint32_t)(k >> 32), c2 = w2, c3 = w3;
        philox4x32_10(c0, c1, c2, c3, k0, k1);
        uint64_t r = ((uint64_t)c0 << 32) | c1;
        int site = (int)__umul64hi(r, (uint64_t)N);
        int cur = sp[site];
        unsigned peers = __match_any_sync(0xffffffffu, site);
        bool first = (peers & lt_mask) == 0;
        bool take = first && cur == kFe;
        unsigned acc = __ballot_sync(0xffffffffu, take);
        int rank = __popc(acc & lt_mask);
        long long q = placed + rank;
        if (take && q < total) {
            int species;
            long long qq = q;
            if (qq < cnt[0]) species = kVac;
            else if ((qq -= cnt[0]) < cnt[1]) species = 1;
            else if ((qq -= cnt[1]) < cnt[2]) species = 2;
            else species = 3;
            sp[site] = (uint8_t)species;
            if (species == kVac) V.vac_pos[q] = site;
        }
        placed += __popc(acc);
        kb += 32;
        __syncwarp();
    }
}

// Whole-batch state load: patch clock and counter from the io staging area
// ([t_hi n][t_lo n][n_events n]), restart displacements, and validate each
// voxel's lattice (codes <= 4, vacancy count, vac_pos names distinct vacancy
// sites).  A voxel that fails gets status EINVAL and is skipped by the
// kernels; one that passes gets status OK.
__global__ void batch_load_kernel(VoxelDev* vox, const double* io, int n, int has_t, int has_n) {
    __shared__ int bad, nvac;
    VoxelDev& V = vox[blockIdx.x];
    if (threadIdx.x == 0) { bad = 0; nvac = 0; }
    __syncthreads();
    int local = 0, lbad = 0;
    for (int i = threadIdx.x; i < V.N; i += blockDim.x) {
        int s = V.species[i];
        lbad |= s > kVac;
        local += s == kVac;
    }
    for (int q = threadIdx.x; q < V.nv; q += blockDim.x) {
        int p = V.vac_pos[q];
        if (p < 0 || p >= V.N || V.species[p] != kVac) lbad = 1;
        for (int r = q + 1; r < V.nv; ++r) lbad |= V.vac_pos[r] == p;
    }
    for (int i = threadIdx.x; i < 3 * V.nv; i += blockDim.x) V.vac_disp[i] = 0;
    if (lbad) atomicExch(&bad, 1);
    atomicAdd(&nvac, local);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (has_t) {
            V.t_hi = io[blockIdx.x];
            V.t_lo = io[n + blockIdx.x];
        }
        if (has_n) V.n_events = ((const uint64_t*)io)[2 * n + blockIdx.x];
        V.status = (bad || nvac != V.nv) ? kEINVAL : kOK;
    }
}

// One voxel's state load (lattice validated on the host): clock and counter
// from io ([t_hi, t_lo, n_events]), displacements restarted, status OK.
__global__ void voxel_load_kernel(VoxelDev* V, const double* io) {
    for (int i = threadIdx.x; i < 3 * V->nv; i += blockDim.x) V->vac_disp[i] = 0;
    if (threadIdx.x == 0) {
        V->t_hi = io[0];
        V->t_lo = io[1];
        V->n_events = ((const uint64_t*)io)[2];
        V->status = kOK;
    }
}

cudaError_t launch_voxel_load(VoxelDev* V, const double* io, cudaStream_t st) {
    voxel_load_kernel<<<1, 128, 0, st>>>(V, io);
    return cudaGetLastError();
}

// Whole-batch state read: clock, counter and status of every voxel into io
// ([t_hi n][t_lo n][n_events n][status n as int32]).
__global__ void batch_read_kernel(const VoxelDev* vox, double* io, int n) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        io[v] = vox[v].t_hi;
        io[n + v] = vox[v].t_lo;
        ((uint64_t*)io)[2 * n + v] = vox[v].n_events;
        ((int32_t*)(io + 3 * n))[v] = vox[v].status;
    }
}

// Workload proxy of the dynamic voxel scheduling (Eq. 10) from each voxel's
// current hop rates: one warp per voxel adds its 8 nv rates (float64; lane-
// strided partial sums, then a butterfly, so the order is fixed) and counts
// the admissible hops (rate > 0).  With Gamma_tot the sum and M the count,
// W = Gamma_tot / nu, and E = -ln(W / M) / beta is the barrier that gives each
// of the M admissible hops the voxel's mean rate, so W = M exp(-beta E).
// io[v] = W, io[n + v] = M, io[2n + v] = E (+inf when M = 0 or Gamma_tot = 0).
__global__ void proxy_kernel(const VoxelDev* vox, const ModelDev* M, double* io, int n) {
    const int lane = threadIdx.x & 31;
    const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (v >= n) return;
    const VoxelDev& V = vox[v];
    double s = 0.0;
    int m = 0;
    for (int i = lane; i < 8 * V.nv; i += 32) {
        const double g = V.rates[i];
        s += g;
        m += g > 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        m += __shfl_xor_sync(0xffffffffu, m, o);
    }
    if (lane == 0) {
        const double W = s / M->nu;
        io[v] = W;
        io[n + v] = (double)m;
        io[2 * n + v] = (m > 0 && s > 0.0) ? -log(W / (double)m) / V.beta : __longlong_as_double(0x7ff0000000000000ll);
    }
}

cudaError_t launch_proxy(const VoxelDev* vox, const ModelDev* M, double* io, int n, cudaStream_t st) {
    proxy_kernel<<<(n + 3) / 4, 128, 0, st>>>(vox, M, io, n);
    return cudaGetLastError();
}

cudaError_t launch_batch_load(VoxelDev* vox, const double* io, int n, int has_t, int has_n, cudaStream_t st) {
    batch_load_kernel<<<n, 256, 0, st>>>(vox, io, n, has_t, has_n);
    return cudaGetLastError();
}

cudaError_t launch_batch_read(const VoxelDev* vox, double* io, int n, cudaStream_t st) {
    batch_read_kernel<<<(n + 127) / 128, 128, 0, st>>>(vox, io, n);
    return cudaGetLastError();
}

void launch_setup_model(ModelDev* M, int32_t* batch_status, int has_eam, int n_rho, cudaStream_t st) {
    int blocks = has_eam ? (4 * n_rho + 255) / 256 : 1;
    if (blocks < 1) blocks = 1;
    setup_model_kernel<<<blocks, 256, 0, st>>>(M, batch_status);
}

void launch_place(VoxelDev* vox, int n_vox, const int32_t* list, cudaStream_t st) {
    int threads = 128;
    int blocks = (n_vox * 32 + threads - 1) / threads;
    place_kernel<<<blocks, threads, 0, st>>>(vox, n_vox, list);
}

}  // namespace akmc
