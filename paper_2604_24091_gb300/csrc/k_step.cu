// k_step.cu -- the AKMC hot path: incremental rate refresh (a2-a5), event
// selection (a6), swap and density update (a7), refresh of affected vacancies
// (a8) and the compensated clock (a9), as one persistent kernel that steps a
// whole voxel per CTA, plus the full rebuild used by akmc_compute_rates.
//
// One CTA owns one voxel at a time and runs all of its requested events; the
// voxel's rates, rate tree and vacancy coordinates live in shared memory while
// it is resident.  Rating the 8 hops of one vacancy is done by warps: warp k
// (mod the CTA's warp count) rates hop k with a fixed lane -> term mapping and
// a fixed shuffle reduction, so results do not depend on the launch shape.
#include "akmc_device.cuh"
#include "akmc_launch.h"

namespace akmc {

struct __align__(16) StepShared {
    double E0[4];
    double nu;
    double inv_knot;
    double phi_d[10][8];
    long long phi_q[10][8];
    const Cubic64* Fd;
    const float4* Ff;
    const long long* Fq;
    int32_t eps_q[2][25];
    int32_t fq[5][8];
    int32_t sph[64];
    int32_t off[160];
    uint32_t ent[8][80];
    int32_t mk[8];
    int32_t n_rho, shift, cur_model, vid;
    float inv_knot_f;
    VoxelDev v;
    uint64_t target;
    // staging of one vacancy's read set
    int32_t srho[160];
    uint8_t ssp[160];
    double hop_de[8];
    int32_t hop_A[8];
    int32_t hop_bad[8];
    // current event
    double R, u2, t_hi, t_lo;
    uint64_t n;
    int32_t stop, numeric, n_aff;
    int32_t slot, dir, A;
    int32_t wX, wY, wZ, mX, mY, mZ;
};

struct Dyn {
    double* tree;
    double* rates;
    double* dE;
    int32_t* pos;
    int32_t* X;
    int32_t* Y;
    int32_t* Z;
    int32_t* disp;
    int32_t* aff;
    uint8_t* hop_sp;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__device__ __forceinline__ Dyn carve(unsigned char* base, int max_nv, int max_P) {
    Dyn d;
    size_t o = 0;
    d.tree = (double*)(base + o);   o = align16(o + sizeof(double) * 2 * max_P);
    d.rates = (double*)(base + o);  o = align16(o + sizeof(double) * 8 * max_nv);
    d.dE = (double*)(base + o);     o = align16(o + sizeof(double) * 8 * max_nv);
    d.pos = (int32_t*)(base + o);   o = align16(o + sizeof(int32_t) * max_nv);
    d.X = (int32_t*)(base + o);     o = align16(o + sizeof(int32_t) * max_nv);
    d.Y = (int32_t*)(base + o);     o = align16(o + sizeof(int32_t) * max_nv);
    d.Z = (int32_t*)(base + o);     o = align16(o + sizeof(int32_t) * max_nv);
    d.disp = (int32_t*)(base + o);  o = align16(o + sizeof(int32_t) * 3 * max_nv);
    d.aff = (int32_t*)(base + o);   o = align16(o + sizeof(int32_t) * max_nv);
    d.hop_sp = (uint8_t*)(base + o);
    return d;
}

size_t step_dyn_smem(int max_nv, int max_P) {
    size_t o = 0;
    o = align16(o + sizeof(double) * 2 * max_P);
    o = align16(o + sizeof(double) * 8 * max_nv);
    o = align16(o + sizeof(double) * 8 * max_nv);
    for (int i = 0; i < 4; ++i) o = align16(o + sizeof(int32_t) * max_nv);
    o = align16(o + sizeof(int32_t) * 3 * max_nv);
    o = align16(o + sizeof(int32_t) * max_nv);
    o = align16(o + 8 * max_nv);
    return o;
}

template <int NW>
__device__ void load_model(StepShared& S, const ModelDev* M) {
    const int tid = threadIdx.x;
    for (int i = tid; i < 50; i += NW * 32) S.eps_q[i / 25][i % 25] = M->eps_q[i / 25][i % 25];
    for (int i = tid; i < 40; i += NW * 32) S.fq[i / 8][i % 8] = M->fq[i / 8][i % 8];
    for (int i = tid; i < 80; i += NW * 32) {
        S.phi_d[i / 8][i % 8] = M->phi_d[i / 8][i % 8];
        S.phi_q[i / 8][i % 8] = M->phi_q[i / 8][i % 8];
    }
    if (tid < 4) S.E0[tid] = M->E0[tid];
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
    }
}

// Stencil tables of the voxel's energy model (reloaded only when it changes).
template <int NW>
__device__ void load_tables(StepShared& S, const Tables* T, int model) {
    const int tid = threadIdx.x;
    if (S.cur_model == model) return;   // uniform: read after a barrier
    __syncthreads();
    if (model == 0) {
        for (int i = tid; i < 64; i += NW * 32) S.off[i] = T->pair_off[i];
        for (int i = tid; i < 8 * 32; i += NW * 32) S.ent[i / 32][i % 32] = T->pair_ent[i / 32][i % 32];
        if (tid < 8) S.mk[tid] = T->pair_mk[tid];
    } else {
        for (int i = tid; i < 160; i += NW * 32) S.off[i] = T->eam_off[i];
        for (int i = tid; i < 8 * 80; i += NW * 32) S.ent[i / 80][i % 80] = T->eam_ent[i / 80][i % 80];
        if (tid < 8) S.mk[tid] = T->eam_mk[tid];
        for (int i = tid; i < 64; i += NW * 32) S.sph[i] = T->sph_off[i];
    }
    __syncthreads();
    if (tid == 0) S.cur_model = model;
    __syncthreads();
}

// Embedding function on the fixed-point density r: knot k = r >> shift,
// t = (r - k*2^shift) 2^-shift (exact).  Outside the table: clamp, flag.
__device__ __forceinline__ void embed_split(const StepShared& S, int a, int r, long long& kq, float& p,
                                            int& bad) {
    const int last = S.n_rho - 1;
    int k = r >> S.shift;
    if (r < 0 || k > last || (k == last && (r & ((1 << S.shift) - 1)))) bad = 1;
    k = min(max(k, 0), last - 1);
    float t = (float)(r - (k << S.shift)) * S.inv_knot_f;
    float4 c = __ldg(&S.Ff[a * last + k]);
    p = t * (c.x + t * (c.y + t * c.z));
    kq = __ldg(&S.Fq[a * S.n_rho + k]);
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

// (a2)-(a5) Rates of the 8 hops of vacancy q, its leaf sum and tree path.
template <int NW>
__device__ void refresh(StepShared& S, const Dyn& D, int q) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = S.v.L, M2 = 2 * L;
    const int X = D.X[q], Y = D.Y[q], Z = D.Z[q];
    const bool eam = S.v.model == 1;
    const int U = eam ? kEamU : kPairU;
    // gather the read set
    for (int u = tid; u < U; u += NW * 32) {
        int o = S.off[u];
        int s = site_index(wrap_coord(X + off_dx(o), M2), wrap_coord(Y + off_dy(o), M2),
                           wrap_coord(Z + off_dz(o), M2), L);
        S.ssp[u] = S.v.species[s];
        if (eam) S.srho[u] = S.v.rho[s];
    }
    __syncthreads();
    for (int k = warp; k < 8; k += NW) {
        const int A = S.ssp[S.mk[k]];
        if (A == kVac) {
            if (lane == 0) { S.hop_A[k] = kVac; S.hop_de[k] = 0.0; S.hop_bad[k] = 0; }
            continue;
        }
        if (!eam) {
            // (a2) dE = sum over the 13 bonds of w (V -> A) and 13 bonds of m (A -> V),
            // exact integer arithmetic in units of 2^-24 eV.
            int acc = 0;
            if (lane < kPairE) {
                uint32_t e = S.ent[k][lane];
                int idx = e & 0xff, sh = (e >> 8) & 1, side = (e >> 9) & 1;
                int x = S.ssp[idx];
                int t = S.eps_q[sh][A * 5 + x] - S.eps_q[sh][kVac * 5 + x];
                acc = side ? -t : t;
            }
            acc = warp_sum(acc);
            if (lane == 0) { S.hop_de[k] = (double)acc * 0x1p-24; S.hop_A[k] = A; S.hop_bad[k] = 0; }
        } else if (S.v.precision == 1) {
            // (a3) split precision: knot values and pair terms exact in 2^-40 eV,
            // the Hermite polynomial part in FP32, assembled in FP64.
            long long aq = 0;
            float af = 0.f;
            int bad = 0;
            for (int j = lane; j < kEamE; j += 32) {
                uint32_t e = S.ent[k][j];
                int a, r0, r1;
                if (e >> 14) {
                    a = A;
                    r0 = S.srho[S.mk[k]];
                    r1 = S.srho[0] - S.fq[A][1];
                } else {
                    int idx = e & 0xff, sip = (e >> 8) & 7, sim = (e >> 11) & 7;
                    a = S.ssp[idx];
                    if (a == kVac) continue;
                    r0 = S.srho[idx];
                    r1 = r0 + S.fq[A][sip] - S.fq[A][sim];
                    int pi = pair_index(A, a);
                    aq += S.phi_q[pi][sip] - S.phi_q[pi][sim];
                }
                long long q0, q1;
                float p0, p1;
                embed_split(S, a, r1, q1, p1, bad);
                embed_split(S, a, r0, q0, p0, bad);
                aq += q1 - q0;
                af += p1 - p0;
            }
            aq = warp_sum(aq);
            af = warp_sum(af);
            bad = __any_sync(0xffffffffu, bad);
            if (lane == 0) {
                S.hop_de[k] = (double)aq * 0x1p-40 + (double)af;
                S.hop_A[k] = A;
                S.hop_bad[k] = bad;
            }
        } else {
            // (a3) FP64 throughout.
            double acc = 0.0;
            int bad = 0;
            for (int j = lane; j < kEamE; j += 32) {
                uint32_t e = S.ent[k][j];
                int a, r0, r1;
                double ph = 0.0;
                if (e >> 14) {
                    a = A;
                    r0 = S.srho[S.mk[k]];
                    r1 = S.srho[0] - S.fq[A][1];
                } else {
                    int idx = e & 0xff, sip = (e >> 8) & 7, sim = (e >> 11) & 7;
                    a = S.ssp[idx];
                    if (a == kVac) continue;
                    r0 = S.srho[idx];
                    r1 = r0 + S.fq[A][sip] - S.fq[A][sim];
                    int pi = pair_index(A, a);
                    ph = S.phi_d[pi][sip] - S.phi_d[pi][sim];
                }
                acc += (embed_fp64(S, a, r1, bad) - embed_fp64(S, a, r0, bad)) + ph;
            }
            acc = warp_sum(acc);
            bad = __any_sync(0xffffffffu, bad);
            if (lane == 0) { S.hop_de[k] = acc; S.hop_A[k] = A; S.hop_bad[k] = bad; }
        }
    }
    __syncthreads();
    // (a4) barriers and rates of the 8 hops in lanes 0..7 of warp 0, (a5) the
    // vacancy sum ((g0+g1)+(g2+g3))+((g4+g5)+(g6+g7)) and its tree path.
    if (warp == 0 && lane < 8) {
        const int A = S.hop_A[lane];
        const double de = S.hop_de[lane];
        int bad = S.hop_bad[lane];
        double g = 0.0;
        if (A != kVac) {
            double Ea = fmax(fmax(0.0, de), S.E0[A] + 0.5 * de);
            g = S.nu * exp(-(Ea * S.v.beta));
            if (!isfinite(g)) bad = 1;
        }
        D.rates[8 * q + lane] = g;
        D.dE[8 * q + lane] = de;
        D.hop_sp[8 * q + lane] = (uint8_t)A;
        double s1 = g + __shfl_xor_sync(0xffu, g, 1);
        double s2 = s1 + __shfl_xor_sync(0xffu, s1, 2);
        double s3 = s2 + __shfl_xor_sync(0xffu, s2, 4);
        bad = __any_sync(0xffu, bad);
        if (lane == 0) {
            const int P = S.v.P;
            D.tree[P + q] = s3;
            for (int i = (P + q) >> 1; i >= 1; i >>= 1) D.tree[i] = D.tree[2 * i] + D.tree[2 * i + 1];
            if (bad) S.numeric = 1;
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
    if (tid == 0) {
        S.t_hi = V.t_hi;
        S.t_lo = V.t_lo;
        S.n = V.n_events;
        S.stop = 0;
        S.numeric = 0;
    }
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

// Events of the resident voxel (a6 -> a7 -> a9 -> a8), target of them at most.
template <int NW>
__device__ void run_events(StepShared& S, const Dyn& D, uint64_t target) {
    const int tid = threadIdx.x;
    const int clock_tid = NW > 1 ? 32 : 0;
    const int L = S.v.L, M2 = 2 * L;
    const bool eam = S.v.model == 1;
    const int reach = eam ? 8 : 4;
    for (uint64_t done = 0; done < target; ++done) {
        // (a6) select with u1 * R; (a7) swap; bookkeeping.
        if (tid == 0) {
            const double R = D.tree[1];
            if (!(R > 0.0)) {
                S.stop = 1;
                S.v.status = kETRAPPED;
            } else {
                double u1, u2;
                event_uniforms(S.v.seed, S.v.uid, S.n, u1, u2);
                double t = u1 * R;
                const int P = S.v.P;
                int node = 1;
                while (node < P) {
                    double l = D.tree[2 * node], r = D.tree[2 * node + 1];
                    if (t < l || r == 0.0) {
                        node = 2 * node;
                    } else {
                        t -= l;
                        node = 2 * node + 1;
                    }
                }
                const int slot = node - P;
                const double* g = D.rates + 8 * slot;
                const double a01 = g[0] + g[1], a23 = g[2] + g[3], a45 = g[4] + g[5], a67 = g[6] + g[7];
                const double b0 = a01 + a23, b1 = a45 + a67;
                int d = 0;
                if (!(t < b0 || b1 == 0.0)) { t -= b0; d = 4; }
                double l2 = d ? a45 : a01, r2 = d ? a67 : a23;
                if (!(t < l2 || r2 == 0.0)) { t -= l2; d += 2; }
                double l3 = g[d], r3 = g[d + 1];
                if (!(t < l3 || r3 == 0.0)) { d += 1; }
                const int dx = (d & 1) ? -1 : 1, dy = (d & 2) ? -1 : 1, dz = (d & 4) ? -1 : 1;
                const int wX = D.X[slot], wY = D.Y[slot], wZ = D.Z[slot];
                const int mX = wrap_coord(wX + dx, M2), mY = wrap_coord(wY + dy, M2),
                          mZ = wrap_coord(wZ + dz, M2);
                const int w = D.pos[slot];
                const int m = site_index(mX, mY, mZ, L);
                const int A = D.hop_sp[8 * slot + d];
                S.v.species[w] = (uint8_t)A;
                S.v.species[m] = (uint8_t)kVac;
                D.pos[slot] = m;
                D.X[slot] = mX;
                D.Y[slot] = mY;
                D.Z[slot] = mZ;
                D.disp[3 * slot + 0] += dx;
                D.disp[3 * slot + 1] += dy;
                D.disp[3 * slot + 2] += dz;
                if (S.v.log_cap > 0) S.v.log[S.n % (uint64_t)S.v.log_cap] = 8 * slot + d;
                S.n += 1;
                S.R = R;
                S.u2 = u2;
                S.slot = slot;
                S.dir = d;
                S.A = A;
                S.wX = wX; S.wY = wY; S.wZ = wZ;
                S.mX = mX; S.mY = mY; S.mZ = mZ;
                S.n_aff = 0;
            }
        }
        __syncthreads();
        if (S.stop) break;
        // (a9) dt = -ln(u2)/R, Neumaier-compensated (t_hi, t_lo).
        if (tid == clock_tid) {
            const double dt = -log(S.u2) / S.R;
            const double s = S.t_hi + dt;
            if (fabs(S.t_hi) >= fabs(dt))
                S.t_lo += (S.t_hi - s) + dt;
            else
                S.t_lo += (dt - s) + S.t_hi;
            S.t_hi = s;
        }
        // (a7) EAM densities: rho_i += f_A(r_iw) over S(w), -= f_A(r_im) over S(m).
        if (eam) {
            for (int i = tid; i < 2 * kSph; i += NW * 32) {
                const int side = i >= kSph;
                const int o = S.sph[side ? i - kSph : i];
                const int cX = side ? S.mX : S.wX, cY = side ? S.mY : S.wY, cZ = side ? S.mZ : S.wZ;
                const int s = site_index(wrap_coord(cX + off_dx(o), M2), wrap_coord(cY + off_dy(o), M2),
                                         wrap_coord(cZ + off_dz(o), M2), L);
                const int f = S.fq[S.A][off_extra(o)];
                atomicAdd(&S.v.rho[s], side ? -f : f);
            }
        }
        // (a8) vacancies whose read set may contain a changed site: the moved
        // one and every vacancy within `reach` half units of w per axis.
        for (int q = tid; q < S.v.nv; q += NW * 32) {
            bool hit = q == S.slot;
            if (!hit) {
                int ddx = D.X[q] - S.wX, ddy = D.Y[q] - S.wY, ddz = D.Z[q] - S.wZ;
                ddx = ddx >= L ? ddx - M2 : (ddx < -L ? ddx + M2 : ddx);
                ddy = ddy >= L ? ddy - M2 : (ddy < -L ? ddy + M2 : ddy);
                ddz = ddz >= L ? ddz - M2 : (ddz < -L ? ddz + M2 : ddz);
                hit = abs(ddx) <= reach && abs(ddy) <= reach && abs(ddz) <= reach;
            }
            if (hit) D.aff[atomicAdd(&S.n_aff, 1)] = q;
        }
        __syncthreads();
        const int n_aff = S.n_aff;
        for (int i = 0; i < n_aff; ++i) refresh<NW>(S, D, D.aff[i]);
        if (S.numeric) {
            if (tid == 0) S.v.status = kENUMERIC;
            break;
        }
    }
    __syncthreads();
}

template <int NW>
__global__ void __launch_bounds__(NW * 32) step_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    __shared__ StepShared S;
    const Dyn D = carve(dyn_raw, a.max_nv, a.max_P);
    load_model<NW>(S, a.model);
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
            load_tables<NW>(S, a.tab, S.v.model);
            load_voxel_state<NW>(S, D);
            __syncthreads();
            run_events<NW>(S, D, S.target);
            store_voxel_state<NW>(S, D, &a.vox[vid]);
        }
        __syncthreads();
    }
}

// Full rebuild of one voxel per CTA: every vacancy's rates, then the tree
// (leaf path updates in slot order leave every node = left + right of its
// final children).
template <int NW>
__global__ void __launch_bounds__(NW * 32) rebuild_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    __shared__ StepShared S;
    const Dyn D = carve(dyn_raw, a.max_nv, a.max_P);
    load_model<NW>(S, a.model);
    if (threadIdx.x == 0) S.v = a.vox[blockIdx.x];
    __syncthreads();
    if (S.v.status == kEINVAL) return;   // placement failed; uniform
    load_tables<NW>(S, a.tab, S.v.model);
    load_voxel_state<NW>(S, D);
    for (int i = threadIdx.x; i < 2 * S.v.P; i += NW * 32) D.tree[i] = 0.0;
    __syncthreads();
    for (int q = 0; q < S.v.nv; ++q) refresh<NW>(S, D, q);
    if (threadIdx.x == 0 && S.numeric) S.v.status = kENUMERIC;
    __syncthreads();
    store_voxel_state<NW>(S, D, &a.vox[blockIdx.x]);
}

template <int NW>
static cudaError_t set_smem(const void* fn, size_t dyn) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

cudaError_t launch_step(const BatchArgs& a, int warps, int grid, cudaStream_t st) {
    size_t dyn = step_dyn_smem(a.max_nv, a.max_P);
    cudaError_t e = cudaSuccess;
    switch (warps) {
#define AKMC_CASE(W)                                                              \
    case W:                                                                       \
        e = set_smem<W>((const void*)step_kernel<W>, dyn);                        \
        if (e != cudaSuccess) return e;                                           \
        step_kernel<W><<<grid, W * 32, dyn, st>>>(a);                             \
        break;
        AKMC_CASE(1) AKMC_CASE(2) AKMC_CASE(4) AKMC_CASE(8)
#undef AKMC_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rebuild(const BatchArgs& a, int warps, cudaStream_t st) {
    size_t dyn = step_dyn_smem(a.max_nv, a.max_P);
    cudaError_t e = cudaSuccess;
    switch (warps) {
#define AKMC_CASE(W)                                                              \
    case W:                                                                       \
        e = set_smem<W>((const void*)rebuild_kernel<W>, dyn);                     \
        if (e != cudaSuccess) return e;                                           \
        rebuild_kernel<W><<<a.n_vox, W * 32, dyn, st>>>(a);                       \
        break;
        AKMC_CASE(1) AKMC_CASE(2) AKMC_CASE(4) AKMC_CASE(8)
#undef AKMC_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int step_occupancy(int warps, int max_nv, int max_P) {
    size_t dyn = step_dyn_smem(max_nv, max_P);
    int n = 0;
    switch (warps) {
        case 1: set_smem<1>((const void*)step_kernel<1>, dyn);
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<1>, 32, dyn); break;
        case 2: set_smem<2>((const void*)step_kernel<2>, dyn);
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<2>, 64, dyn); break;
        case 4: set_smem<4>((const void*)step_kernel<4>, dyn);
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<4>, 128, dyn); break;
        case 8: set_smem<8>((const void*)step_kernel<8>, dyn);
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<8>, 256, dyn); break;
        default: break;
    }
    return n;
}

}  // namespace akmc
