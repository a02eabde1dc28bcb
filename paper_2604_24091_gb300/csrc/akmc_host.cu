// akmc_host.cu -- host implementation of the C ABI declared in include/akmc.h.
// Validates inputs, lays a batch out in the caller's workspace, uploads the
// model and descriptors, and launches the kernels on the caller's stream.
#include <akmc.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "akmc_device.cuh"
#include "akmc_launch.h"

using namespace akmc;

namespace {

thread_local std::string g_err;

akmc_status fail(akmc_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define AKMC_CUDA(call)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(AKMC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));           \
    } while (0)

// ---------------------------------------------------------------- stencil tables

struct Off3 { int dx, dy, dz; };
bool operator==(const Off3& a, const Off3& b) { return a.dx == b.dx && a.dy == b.dy && a.dz == b.dz; }

int shell_of(const Off3& o) {
    switch (o.dx * o.dx + o.dy * o.dy + o.dz * o.dz) {
        case 3: return 1;
        case 4: return 2;
        case 8: return 3;
        case 11: return 4;
        case 12: return 5;
        default: return 0;
    }
}

bool same_parity(int dx, int dy, int dz) {
    int a = dx & 1, b = dy & 1, c = dz & 1;
    return a == b && b == c;
}

Tables make_tables() {
    Tables T;
    std::memset(&T, 0, sizeof T);
    std::vector<Off3> sph;
    for (int want = 1; want <= 5; ++want)
        for (int dz = -4; dz <= 4; ++dz)
            for (int dy = -4; dy <= 4; ++dy)
                for (int dx = -4; dx <= 4; ++dx) {
                    Off3 o{dx, dy, dz};
                    if (!same_parity(dx, dy, dz) || shell_of(o) != want) continue;
                    sph.push_back(o);
                }
    for (size_t i = 0; i < sph.size(); ++i)
        T.sph_off[i] = off_pack(sph[i].dx, sph[i].dy, sph[i].dz, shell_of(sph[i]));
    std::vector<Off3> n12(sph.begin(), sph.begin() + 14);
    Off3 dirs[8];
    for (int k = 0; k < 8; ++k) dirs[k] = Off3{(k & 1) ? -1 : 1, (k & 2) ? -1 : 1, (k & 4) ? -1 : 1};
    auto plus = [](Off3 a, Off3 b) { return Off3{a.dx + b.dx, a.dy + b.dy, a.dz + b.dz}; };
    auto minus = [](Off3 a, Off3 b) { return Off3{a.dx - b.dx, a.dy - b.dy, a.dz - b.dz}; };
    auto index_in = [](std::vector<Off3>& U, Off3 o) {
        for (size_t i = 0; i < U.size(); ++i)
            if (U[i] == o) return (int)i;
        U.push_back(o);
        return (int)U.size() - 1;
    };
    auto contains = [](const std::vector<Off3>& U, Off3 o) {
        for (const Off3& u : U)
            if (u == o) return true;
        return false;
    };
    // pair model: bonds of w = the vacancy (offset 0) and of m_k = d_k
    std::vector<Off3> U{Off3{0, 0, 0}};
    for (const Off3& o : n12) index_in(U, o);
    for (int k = 0; k < 8; ++k)
        for (const Off3& o : n12) index_in(U, plus(dirs[k], o));
    for (int k = 0; k < 8; ++k) {
        T.pair_mk[k] = index_in(U, dirs[k]);
        int e = 0;
        for (const Off3& o : n12) {
            if (o == dirs[k]) continue;
            T.pair_ent[k][e++] = (uint32_t)index_in(U, o) | ((uint32_t)(shell_of(o) - 1) << 8);
        }
        for (const Off3& o : n12) {
            Off3 j = plus(dirs[k], o);
            if (j == Off3{0, 0, 0}) continue;
            T.pair_ent[k][e++] = (uint32_t)index_in(U, j) | ((uint32_t)(shell_of(o) - 1) << 8) | (1u << 9);
        }
    }
    for (size_t i = 0; i < U.size(); ++i) T.pair_off[i] = off_pack(U[i].dx, U[i].dy, U[i].dz, 0);
    // EAM: union of S(0) and S(d_k)
    std::vector<Off3> E{Off3{0, 0, 0}};
    for (const Off3& o : sph) index_in(E, o);
    for (int k = 0; k < 8; ++k)
        for (const Off3& o : sph) index_in(E, plus(dirs[k], o));
    for (int k = 0; k < 8; ++k) {
        T.eam_mk[k] = index_in(E, dirs[k]);
        std::vector<Off3> aff;
        for (const Off3& o : sph)
            if (!(o == dirs[k]) && !contains(aff, o)) aff.push_back(o);
        for (const Off3& o : sph) {
            Off3 i = plus(dirs[k], o);
            if (!(i == Off3{0, 0, 0}) && !contains(aff, i)) aff.push_back(i);
        }
        int e = 0;
        for (const Off3& i : aff) {
            int sip = contains(sph, i) ? shell_of(i) : 0;
            Off3 im = minus(i, dirs[k]);
            int sim = contains(sph, im) ? shell_of(im) : 0;
            T.eam_ent[k][e++] = (uint32_t)index_in(E, i) | ((uint32_t)sip << 8) | ((uint32_t)sim << 11);
        }
        T.eam_ent[k][e++] = 1u << 14;   // the moving atom's own embedding term
    }
    for (size_t i = 0; i < E.size(); ++i) T.eam_off[i] = off_pack(E[i].dx, E[i].dy, E[i].dz, 0);
    for (int small = 0; small < 2; ++small)
        for (size_t u = 0; u < E.size(); ++u)
            for (int k = 0; k < 8; ++k) {
                Off3 uw = plus(E[u], dirs[k]);   // u - w with w = m - d_k
                if (small) {
                    auto img = [](int c) { return c > 4 ? c - 8 : (c <= -4 ? c + 8 : c); };
                    uw = Off3{img(uw.dx), img(uw.dy), img(uw.dz)};
                }
                int sw = contains(sph, uw) ? shell_of(uw) : 0;
                int sm = contains(sph, E[u]) ? shell_of(E[u]) : 0;
                T.eam_dsh[small][u][k] = (uint8_t)((sw << 3) | sm);
            }
    auto region = [&](const std::vector<Off3>& Un, int32_t* roff, uint16_t* ridx, int ustride, int32_t& nreg,
                      int32_t* rc) {
        std::vector<Off3> R;
        for (int k = 0; k < 8; ++k)
            for (const Off3& u : Un) index_in(R, plus(dirs[k], u));
        for (size_t i = 0; i < R.size(); ++i) roff[i] = off_pack(R[i].dx, R[i].dy, R[i].dz, 0);
        for (int k = 0; k < 8; ++k)
            for (size_t u = 0; u < Un.size(); ++u) ridx[k * ustride + u] = (uint16_t)index_in(R, plus(dirs[k], Un[u]));
        nreg = (int32_t)R.size();
        for (int k = 0; k < 8; ++k) rc[k] = index_in(R, dirs[k]);
        rc[8] = index_in(R, Off3{0, 0, 0});
        nreg = (int32_t)R.size();
    };
    region(U, T.pair_roff, &T.pair_ridx[0][0], 64, T.pair_nreg, T.pair_rc);
    region(E, T.eam_roff, &T.eam_ridx[0][0], 160, T.eam_nreg, T.eam_rc);
    return T;
}

const Tables& tables() {
    static Tables T = make_tables();
    return T;
}

}  // namespace

const Tables& akmc::host_tables() { return tables(); }
void akmc::set_last_error(const char* msg) { g_err = msg; }

namespace {

// ---------------------------------------------------------------- validation

int next_pow2(int n) {
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

int rho_shift_of(double h) {
    if (!(h > 0.0) || !std::isfinite(h)) return -1;
    int e = 0;
    while (h < 1.0 && e <= kRhoBits) { h *= 2.0; ++e; }
    if (h != 1.0 || e > kRhoBits) return -1;
    return kRhoBits - e;
}

bool all_finite(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

void species_counts(const akmc_voxel_desc& d, int32_t cnt[4]) {
    double N = 2.0 * d.L * (double)d.L * d.L;
    cnt[0] = d.n_vac;
    for (int s = 0; s < 3; ++s) cnt[s + 1] = (int32_t)std::floor(d.frac[s] * N + 0.5);
}

akmc_status validate(const akmc_voxel_desc* descs, int32_t n, const akmc_model* m, int32_t log_cap,
                     bool* has_eam) {
    if (!descs || n < 1) return fail(AKMC_EINVAL, "need at least one voxel descriptor");
    if (!m) return fail(AKMC_EINVAL, "model is NULL");
    if (log_cap < 0) return fail(AKMC_EINVAL, "event_log_capacity < 0");
    *has_eam = false;
    for (int32_t v = 0; v < n; ++v) {
        const akmc_voxel_desc& d = descs[v];
        if (d.model != AKMC_PAIR && d.model != AKMC_EAM) return fail(AKMC_EINVAL, "voxel %d: bad model", v);
        if (d.precision != AKMC_FP64 && d.precision != AKMC_SPLIT)
            return fail(AKMC_EINVAL, "voxel %d: bad precision", v);
        int Lmin = d.model == AKMC_PAIR ? 3 : 4;
        if (d.L < Lmin || d.L > 1023) return fail(AKMC_EINVAL, "voxel %d: L=%d out of range", v, d.L);
        if (d.n_vac < 1 || d.n_vac > kMaxNV) return fail(AKMC_EINVAL, "voxel %d: n_vac=%d", v, d.n_vac);
        if (!(d.T > 0.0) || !std::isfinite(d.T)) return fail(AKMC_EINVAL, "voxel %d: bad T", v);
        int32_t cnt[4];
        for (int s = 0; s < 3; ++s)
            if (!(d.frac[s] >= 0.0) || !(d.frac[s] <= 1.0)) return fail(AKMC_EINVAL, "voxel %d: bad frac", v);
        species_counts(d, cnt);
        long long tot = (long long)cnt[0] + cnt[1] + cnt[2] + cnt[3];
        if (tot > 2LL * d.L * d.L * d.L) return fail(AKMC_EINVAL, "voxel %d: more solutes than sites", v);
        if (d.model == AKMC_EAM) *has_eam = true;
    }
    for (int i = 0; i < 25; ++i)
        for (const double* e : {m->eps1, m->eps2}) {
            double q = e[i] * 16777216.0;
            if (!std::isfinite(q) || q != std::floor(q) || std::fabs(q) >= 67108864.0)
                return fail(AKMC_EINVAL, "pair energies must be multiples of 2^-24 eV below 4 eV");
            if (e[i] != e[(i % 5) * 5 + i / 5]) return fail(AKMC_EINVAL, "pair energies must be symmetric");
        }
    if (!all_finite(m->E0, 4) || !(m->nu > 0.0) || !std::isfinite(m->nu))
        return fail(AKMC_EINVAL, "bad E0 or nu");
    for (int a = 0; a < 4; ++a)
        if (!(m->E0[a] >= 0.0 && m->E0[a] < 4.0)) return fail(AKMC_EINVAL, "E0 must lie in [0, 4) eV");
    if (*has_eam) {
        if (m->n_r < 2 || m->n_rho < 2 || !m->phi_tab || !m->f_tab || !m->F_tab)
            return fail(AKMC_EINVAL, "EAM voxels need phi/f/F tables");
        if (!(m->a > 0.0) || !(m->r_cut > m->a * std::sqrt(3.0)) || !(m->r_cut < 2.0 * m->a))
            return fail(AKMC_EINVAL, "r_cut must lie between the 5th and 6th bcc shells");
        int sh = rho_shift_of(m->rho_h);
        if (sh < 0 || sh > 23) return fail(AKMC_EINVAL, "rho_h must be a power of two in [2^-24, 2^-1]");
        if ((double)(m->n_rho - 1) * std::ldexp(1.0, sh) >= 2147483648.0)
            return fail(AKMC_EINVAL, "embedding table too long for the fixed-point density");
        if (!all_finite(m->phi_tab, 20 * (size_t)m->n_r) || !all_finite(m->f_tab, 8 * (size_t)m->n_r) ||
            !all_finite(m->F_tab, 8 * (size_t)m->n_rho))
            return fail(AKMC_EINVAL, "EAM tables must be finite");
        for (size_t i = 0; i < 8 * (size_t)m->n_rho; i += 2)
            if (std::fabs(m->F_tab[i]) >= 4194304.0) return fail(AKMC_EINVAL, "|F| too large");
    }
    return AKMC_OK;
}

// ---------------------------------------------------------------- layout

constexpr size_t kAlign = 256;
size_t al(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t status = 0, model = 0, tab = 0, vox = 0, targets = 0, order = 0, queue = 0, hist = 0;
    size_t phi_raw = 0, f_raw = 0, F_raw = 0, Fd = 0, Ff = 0, Fq = 0, items = 0;
    size_t labels = 0, sizes = 0, total = 0, ident = 0, sl_done = 0;
    int sl_max_sectors = 0;
    std::vector<size_t> species, rho, pos, disp, rates, dE, hop, tree, log, etab;
    size_t state_begin = 0, state_end = 0, io = 0, reset_list = 0, reset_items = 0;
    size_t b_species = 0, b_pos = 0, b_disp = 0, tot_N = 0, tot_nv = 0;
    std::vector<int4> item_list;       // density tiles (voxels with L > kStripMaxL)
    std::vector<int4> strip_list;      // density strips (voxels with L <= kStripMaxL)
    size_t strips = 0, reset_strips = 0;
    int strip_lmax = 0;
    size_t strip_dyn = 0;              // dynamic shared memory of the strip kernel (batch maximum)
    int max_nv = 1, max_P = 1, win = 0;
    size_t max_N = 0;
    bool has_eam = false;
};

Layout make_layout(const akmc_voxel_desc* d, int32_t n, const akmc_model* m, int32_t log_cap, bool has_eam) {
    Layout Lo;
    Lo.has_eam = has_eam;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = al(o + bytes); return at; };
    Lo.status = take(sizeof(int32_t) * 4);
    Lo.queue = take(sizeof(uint32_t) * 4);
    Lo.hist = take(sizeof(unsigned long long) * 8);
    Lo.model = take(sizeof(ModelDev));
    Lo.tab = take(sizeof(Tables));
    Lo.vox = take(sizeof(VoxelDev) * n);
    Lo.targets = take(sizeof(uint64_t) * n + sizeof(int32_t) * n);   // targets then order
    Lo.order = Lo.targets + sizeof(uint64_t) * n;
    Lo.ident = take(sizeof(int32_t) * n);   // 0, 1, ..., n-1: single-voxel kernel lists
    int nv_max = 1;
    for (int32_t v = 0; v < n; ++v) {
        const int ns = d[v].L / 8;
        Lo.sl_max_sectors = std::max(Lo.sl_max_sectors, ns * ns * ns);
        nv_max = std::max(nv_max, d[v].n_vac);
    }
    // sublattice words: abort word (+3 spare), done[sectors], then stale[vacancies]
    Lo.sl_done = take(sizeof(int32_t) * (4 + (size_t)Lo.sl_max_sectors + (size_t)nv_max));
    if (has_eam) {
        Lo.phi_raw = take(sizeof(double) * 20 * m->n_r);
        Lo.f_raw = take(sizeof(double) * 8 * m->n_r);
        Lo.F_raw = take(sizeof(double) * 8 * m->n_rho);
        Lo.Fd = take(sizeof(Cubic64) * 4 * (m->n_rho - 1));
        Lo.Ff = take(sizeof(float4) * 4 * m->n_rho);   // one zero pad per species at the last knot
        Lo.Fq = take(sizeof(long long) * 4 * m->n_rho);
        for (int32_t v = 0; v < n; ++v) {
            if (d[v].model != AKMC_EAM) continue;
            int L = d[v].L;
            if (L <= kStripMaxL) {
                Lo.strip_lmax = std::max(Lo.strip_lmax, L);
                continue;
            }
            for (int z = 0; z < L; z += kTZ)
                for (int y = 0; y < L; y += kTY)
                    for (int x = 0; x < L; x += kTX) Lo.item_list.push_back(make_int4(v, x, y, z));
        }
        // Strips: density_strip_rows(L) rows per strip (bounded by shared memory
        // and by the 16-byte chunks a thread holds); the z extent tz is the
        // largest of {L, 64, 32, 16, 8} that still gives >= 1024 strips (several waves).
        if (Lo.strip_lmax > 0) {
            const int cand[5] = {1 << 30, 64, 32, 16, 8};
            int tz_cap = 8;
            for (int ci = 0; ci < 5; ++ci) {
                long long cnt = 0;
                for (int32_t v = 0; v < n; ++v) {
                    if (d[v].model != AKMC_EAM || d[v].L > kStripMaxL) continue;
                    const int L = d[v].L, tz = std::min(cand[ci], L), ty = density_strip_rows(L);
                    cnt += (long long)((L + ty - 1) / ty) * ((L + tz - 1) / tz);
                }
                if (cnt >= 1024) {
                    tz_cap = cand[ci];
                    break;
                }
            }
            for (int32_t v = 0; v < n; ++v) {
                if (d[v].model != AKMC_EAM || d[v].L > kStripMaxL) continue;
                const int L = d[v].L, tz = std::min(tz_cap, L), ty = density_strip_rows(L);
                Lo.strip_dyn = std::max(Lo.strip_dyn, density_strip_smem(L));
                for (int z = 0; z < L; z += tz)
                    for (int y = 0; y < L; y += ty)
                        Lo.strip_list.push_back(make_int4(v, y, z, std::min(tz, L - z) | (ty << 17)));
            }
        }
        Lo.items = take(sizeof(int4) * std::max<size_t>(1, Lo.item_list.size()));
        Lo.reset_items = take(sizeof(int4) * std::max<size_t>(1, Lo.item_list.size()));
        Lo.strips = take(sizeof(int4) * std::max<size_t>(1, Lo.strip_list.size()));
        Lo.reset_strips = take(sizeof(int4) * std::max<size_t>(1, Lo.strip_list.size()));
    }
    Lo.reset_list = take(sizeof(int32_t) * n);
    Lo.io = take(32 * (size_t)n);
    // Per-voxel state, each kind concatenated in voxel order so that whole-batch
    // transfers are single copies.
    Lo.state_begin = o;
    size_t tot_N = 0, tot_rho = 0, tot_nv = 0, tot_P = 0;
    for (int32_t v = 0; v < n; ++v) {
        size_t N = 2 * (size_t)d[v].L * d[v].L * d[v].L;
        int nv = d[v].n_vac, P = next_pow2(nv);
        Lo.max_nv = std::max(Lo.max_nv, nv);
        // a single vacancy in a lattice too small for the one-vacancy fast path
        // (L < 6) takes the general path, whose staging the layout sizes for max_nv > 1
        if (nv == 1 && d[v].L < 6) Lo.max_nv = std::max(Lo.max_nv, 2);
        Lo.max_P = std::max(Lo.max_P, P);
        Lo.win = std::max(Lo.win, window_edge(d[v].L, nv, d[v].model, d[v].precision));
        Lo.max_N = std::max(Lo.max_N, N);
        Lo.species.push_back(tot_N);
        Lo.rho.push_back(d[v].model == AKMC_EAM ? tot_rho : 0);
        Lo.pos.push_back(tot_nv);
        Lo.tree.push_back(tot_P);
        tot_N += N;
        if (d[v].model == AKMC_EAM) tot_rho += N;
        tot_nv += nv;
        tot_P += 2 * (size_t)P;
    }
    Lo.tot_N = tot_N;
    Lo.tot_nv = tot_nv;
    const size_t b_species = take(tot_N), b_rho = take(sizeof(int32_t) * tot_rho);
    const size_t b_pos = take(sizeof(int32_t) * tot_nv), b_disp = take(sizeof(int32_t) * 3 * tot_nv);
    const size_t b_rates = take(sizeof(double) * 8 * tot_nv), b_dE = take(sizeof(double) * 8 * tot_nv);
    const size_t b_hop = take(8 * tot_nv), b_tree = take(sizeof(double) * tot_P);
    const size_t b_log = take(sizeof(int32_t) * (size_t)log_cap * n);
    const size_t b_etab = take(sizeof(double) * kEtab * (size_t)n);
    Lo.b_species = b_species;
    Lo.b_pos = b_pos;
    Lo.b_disp = b_disp;
    for (int32_t v = 0; v < n; ++v) {
        const size_t nv0 = Lo.pos[v];
        Lo.species[v] += b_species;
        Lo.rho[v] = d[v].model == AKMC_EAM ? b_rho + sizeof(int32_t) * Lo.rho[v] : 0;
        Lo.pos[v] = b_pos + sizeof(int32_t) * nv0;
        Lo.disp.push_back(b_disp + sizeof(int32_t) * 3 * nv0);
        Lo.rates.push_back(b_rates + sizeof(double) * 8 * nv0);
        Lo.dE.push_back(b_dE + sizeof(double) * 8 * nv0);
        Lo.hop.push_back(b_hop + 8 * nv0);
        Lo.tree[v] = b_tree + sizeof(double) * Lo.tree[v];
        Lo.log.push_back(log_cap > 0 ? b_log + sizeof(int32_t) * (size_t)log_cap * v : 0);
        Lo.etab.push_back(b_etab + sizeof(double) * kEtab * (size_t)v);
    }
    // 16-byte rows (vector loads and stores) where L % 8 == 0 and both
    // arrays of the voxel start on a 16-byte boundary of the 256-byte aligned
    // workspace.
    for (int4& it : Lo.strip_list) {
        const int v = it.x, L = d[v].L;
        const bool vec = L % 8 == 0 && Lo.species[v] % 16 == 0 && Lo.rho[v] % 16 == 0;
        it.w |= (vec ? 1 : 0) << 16;
    }
    Lo.state_end = o;
    Lo.labels = take(sizeof(int32_t) * Lo.max_N);
    Lo.sizes = take(sizeof(int32_t) * Lo.max_N);
    Lo.total = o;
    return Lo;
}

}  // namespace

struct akmc_batch {
    int32_t n = 0;
    int32_t log_cap = 0;
    char* base = nullptr;
    Layout lo;
    std::vector<akmc_voxel_desc> desc;
    std::vector<VoxelDev> vox_host;    // pointers and constants (device copy is authoritative for state)
    ModelDev model_host{};
    std::vector<double> phi_raw, f_raw, F_raw;
    static constexpr int kStage = 4;   // ring of pinned staging slots: targets + order
    char* staging = nullptr;
    cudaEvent_t staging_done[kStage] = {};
    bool staging_used[kStage] = {};
    int stage = 0;
    bool dirty = false;
    int warps = 4, ctas_per_sm = 0, n_sm = 0, device = 0;
    int occupancy[17] = {};            // CTAs per SM of the step kernel, by warps per CTA

    BatchArgs args() const {
        BatchArgs a;
        a.vox = (VoxelDev*)(base + lo.vox);
        a.model = (const ModelDev*)(base + lo.model);
        a.tab = (const Tables*)(base + lo.tab);
        a.order = (const int32_t*)(base + lo.order);
        a.targets = (const uint64_t*)(base + lo.targets);
        a.queue = (uint32_t*)(base + lo.queue);
        a.batch_status = (int32_t*)(base + lo.status);
        a.n_vox = n;
        a.max_nv = lo.max_nv;
        a.max_P = lo.max_P;
        a.win = lo.win;
        return a;
    }
};

namespace {

akmc_status rebuild(akmc_batch* b, cudaStream_t st) {
    BatchArgs a = b->args();
    if (b->lo.has_eam && (!b->lo.item_list.empty() || !b->lo.strip_list.empty())) {
        cudaError_t e = launch_density(a.vox, a.model, a.tab, (const int4*)(b->base + b->lo.items),
                                       (int)b->lo.item_list.size(), (const int4*)(b->base + b->lo.strips),
                                       (int)b->lo.strip_list.size(), b->lo.strip_dyn, st);
        if (e != cudaSuccess) return fail(AKMC_ECUDA, "density kernel: %s", cudaGetErrorString(e));
    }
    cudaError_t e = launch_rebuild(a, 8, nullptr, 0, st);
    if (e != cudaSuccess) return fail(AKMC_ECUDA, "rebuild kernel: %s", cudaGetErrorString(e));
    b->dirty = false;
    return AKMC_OK;
}

}  // namespace

extern "C" {

const char* akmc_last_error(void) { return g_err.c_str(); }

size_t akmc_workspace_bytes(const akmc_voxel_desc* descs, int32_t n, const akmc_model* model,
                            int32_t log_cap) {
    bool has_eam = false;
    if (validate(descs, n, model, log_cap, &has_eam) != AKMC_OK) return 0;
    return make_layout(descs, n, model, log_cap, has_eam).total;
}

akmc_status akmc_create_batch(const akmc_voxel_desc* descs, int32_t n, const akmc_model* m, int32_t log_cap,
                              void* ws, size_t ws_bytes, akmc_stream stream, akmc_batch** out) {
    if (!out) return fail(AKMC_EINVAL, "out is NULL");
    *out = nullptr;
    bool has_eam = false;
    akmc_status st = validate(descs, n, m, log_cap, &has_eam);
    if (st != AKMC_OK) return st;
    if (!ws) return fail(AKMC_EINVAL, "workspace is NULL");
    if ((uintptr_t)ws % kAlign) return fail(AKMC_EINVAL, "workspace must be 256-byte aligned");
    Layout lo = make_layout(descs, n, m, log_cap, has_eam);
    if (ws_bytes < lo.total)
        return fail(AKMC_ENOMEM, "workspace has %zu bytes, batch needs %zu", ws_bytes, lo.total);
    cudaStream_t s = (cudaStream_t)stream;
    akmc_batch* b = new akmc_batch();
    b->n = n;
    b->log_cap = log_cap;
    b->base = (char*)ws;
    b->lo = lo;
    b->desc.assign(descs, descs + n);
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    b->warps = has_eam ? 8 : 4;
    // model image
    ModelDev& M = b->model_host;
    std::memset(&M, 0, sizeof M);
    for (int i = 0; i < 25; ++i) {
        M.eps_q[0][i] = (int32_t)(m->eps1[i] * 16777216.0);
        M.eps_q[1][i] = (int32_t)(m->eps2[i] * 16777216.0);
    }
    for (int i = 0; i < 4; ++i) {
        M.E0[i] = m->E0[i];
        M.two_E0[i] = 2.0 * m->E0[i];
        M.thr_hi[i] = (int32_t)std::floor(2.0 * m->E0[i] * 16777216.0);
        M.thr_lo[i] = -M.thr_hi[i];
    }
    M.nu = m->nu;
    M.has_eam = has_eam;
    if (has_eam) {
        M.a = m->a;
        M.r_cut = m->r_cut;
        M.rho_h = m->rho_h;
        M.n_r = m->n_r;
        M.n_rho = m->n_rho;
        M.shift = rho_shift_of(m->rho_h);
        M.inv_knot = std::ldexp(1.0, -M.shift);
        b->phi_raw.assign(m->phi_tab, m->phi_tab + 20 * (size_t)m->n_r);
        b->f_raw.assign(m->f_tab, m->f_tab + 8 * (size_t)m->n_r);
        b->F_raw.assign(m->F_tab, m->F_tab + 8 * (size_t)m->n_rho);
        M.phi_tab = (const double*)(b->base + lo.phi_raw);
        M.f_tab = (const double*)(b->base + lo.f_raw);
        M.F_tab = (const double*)(b->base + lo.F_raw);
        M.Fd = (Cubic64*)(b->base + lo.Fd);
        M.Ff = (float4*)(b->base + lo.Ff);
        M.Fq = (long long*)(b->base + lo.Fq);
    }
    // voxel images
    b->vox_host.resize(n);
    for (int32_t v = 0; v < n; ++v) {
        const akmc_voxel_desc& d = descs[v];
        VoxelDev& V = b->vox_host[v];
        std::memset(&V, 0, sizeof V);
        V.L = d.L;
        V.N = 2 * d.L * d.L * d.L;
        V.nv = d.n_vac;
        V.P = next_pow2(d.n_vac);
        V.model = d.model;
        V.precision = d.precision;
        V.status = AKMC_OK;
        V.log_cap = log_cap;
        species_counts(d, V.counts);
        V.beta = 1.0 / (kKB * d.T);
        for (int s = 0; s < 3; ++s) V.frac[s] = d.frac[s];
        V.T = d.T;
        V.seed = d.seed;
        V.uid = d.uid;
        V.species = (uint8_t*)(b->base + lo.species[v]);
        V.rho = d.model == AKMC_EAM ? (int32_t*)(b->base + lo.rho[v]) : nullptr;
        V.vac_pos = (int32_t*)(b->base + lo.pos[v]);
        V.vac_disp = (int32_t*)(b->base + lo.disp[v]);
        V.rates = (double*)(b->base + lo.rates[v]);
        V.dE = (double*)(b->base + lo.dE[v]);
        V.hop_sp = (uint8_t*)(b->base + lo.hop[v]);
        V.tree = (double*)(b->base + lo.tree[v]);
        V.log = log_cap > 0 ? (int32_t*)(b->base + lo.log[v]) : nullptr;
        V.etab = (double*)(b->base + lo.etab[v]);
    }
    const size_t stage_bytes = (sizeof(uint64_t) + sizeof(int32_t)) * n;
    cudaError_t e = cudaMallocHost((void**)&b->staging, stage_bytes * akmc_batch::kStage);
    for (int i = 0; i < akmc_batch::kStage && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&b->staging_done[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        akmc_destroy_batch(b);
        return fail(AKMC_ECUDA, "pinned staging: %s", cudaGetErrorString(e));
    }
    std::memset(b->staging, 0, (sizeof(uint64_t) + sizeof(int32_t)) * n);
    int32_t* order = (int32_t*)(b->staging + sizeof(uint64_t) * n);
    for (int32_t v = 0; v < n; ++v) order[v] = v;
#define AKMC_TRY(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            akmc_destroy_batch(b);                                                             \
            return fail(AKMC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));           \
        }                                                                                      \
    } while (0)
    AKMC_TRY(cudaMemsetAsync(b->base, 0, lo.tab, s));
    AKMC_TRY(cudaMemcpyAsync(b->base + lo.model, &M, sizeof M, cudaMemcpyHostToDevice, s));
    AKMC_TRY(cudaMemcpyAsync(b->base + lo.tab, &tables(), sizeof(Tables), cudaMemcpyHostToDevice, s));
    AKMC_TRY(cudaMemcpyAsync(b->base + lo.vox, b->vox_host.data(), sizeof(VoxelDev) * n,
                             cudaMemcpyHostToDevice, s));
    AKMC_TRY(cudaMemcpyAsync(b->base + lo.targets, b->staging, (sizeof(uint64_t) + sizeof(int32_t)) * n,
                             cudaMemcpyHostToDevice, s));
    std::vector<int32_t> ident(n);
    for (int32_t v = 0; v < n; ++v) ident[v] = v;
    AKMC_TRY(cudaMemcpyAsync(b->base + lo.ident, ident.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    AKMC_TRY(cudaEventRecord(b->staging_done[0], s));
    b->staging_used[0] = true;
    b->stage = 1;
    if (has_eam) {
        AKMC_TRY(cudaMemcpyAsync(b->base + lo.phi_raw, b->phi_raw.data(), sizeof(double) * b->phi_raw.size(),
                                 cudaMemcpyHostToDevice, s));
        AKMC_TRY(cudaMemcpyAsync(b->base + lo.f_raw, b->f_raw.data(), sizeof(double) * b->f_raw.size(),
                                 cudaMemcpyHostToDevice, s));
        AKMC_TRY(cudaMemcpyAsync(b->base + lo.F_raw, b->F_raw.data(), sizeof(double) * b->F_raw.size(),
                                 cudaMemcpyHostToDevice, s));
        if (!lo.item_list.empty())
            AKMC_TRY(cudaMemcpyAsync(b->base + lo.items, lo.item_list.data(), sizeof(int4) * lo.item_list.size(),
                                     cudaMemcpyHostToDevice, s));
        if (!lo.strip_list.empty())
            AKMC_TRY(cudaMemcpyAsync(b->base + lo.strips, lo.strip_list.data(),
                                     sizeof(int4) * lo.strip_list.size(), cudaMemcpyHostToDevice, s));
    }
    AKMC_TRY(cudaMemsetAsync(b->base + lo.state_begin, 0, lo.state_end - lo.state_begin, s));
    launch_setup_model((ModelDev*)(b->base + lo.model), (int32_t*)(b->base + lo.status), has_eam,
                       has_eam ? m->n_rho : 0, s);
    AKMC_TRY(cudaGetLastError());
    launch_place((VoxelDev*)(b->base + lo.vox), n, nullptr, s);
    AKMC_TRY(cudaGetLastError());
    AKMC_TRY(launch_rate_tables((VoxelDev*)(b->base + lo.vox), n, (const ModelDev*)(b->base + lo.model), nullptr, s));
    // The pageable host images above must outlive their copies.
    AKMC_TRY(cudaStreamSynchronize(s));
#undef AKMC_TRY
    st = rebuild(b, s);
    if (st != AKMC_OK) {
        akmc_destroy_batch(b);
        return st;
    }
    *out = b;
    return AKMC_OK;
}

akmc_status akmc_compute_rates(akmc_batch* b, akmc_stream stream) {
    if (!b) return fail(AKMC_EINVAL, "batch is NULL");
    return rebuild(b, (cudaStream_t)stream);
}

akmc_status akmc_set_targets(akmc_batch* b, const uint64_t* n_events, akmc_stream stream) {
    if (!b || !n_events) return fail(AKMC_EINVAL, "batch or n_events is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    {
        // a device (or managed) array: copied on the stream, processing order kept
        cudaPointerAttributes at{};
        const cudaError_t pe = cudaPointerGetAttributes(&at, n_events);
        if (pe != cudaSuccess) cudaGetLastError();
        if (pe == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
            AKMC_CUDA(cudaMemcpyAsync(b->base + b->lo.targets, n_events, sizeof(uint64_t) * b->n,
                                      cudaMemcpyDeviceToDevice, s));
            if (b->occupancy[b->warps] == 0)
                b->occupancy[b->warps] = step_occupancy(b->warps, b->lo.max_nv, b->lo.max_P, b->lo.win);
            return AKMC_OK;
        }
    }
    const int slot = b->stage;
    b->stage = (b->stage + 1) % akmc_batch::kStage;
    if (b->staging_used[slot]) AKMC_CUDA(cudaEventSynchronize(b->staging_done[slot]));
    char* stg = b->staging + (sizeof(uint64_t) + sizeof(int32_t)) * b->n * slot;
    uint64_t* tg = (uint64_t*)stg;
    int32_t* order = (int32_t*)(stg + sizeof(uint64_t) * b->n);
    std::vector<std::pair<double, int32_t>> work(b->n);
    for (int32_t v = 0; v < b->n; ++v) {
        tg[v] = n_events[v];
        double cost = (double)n_events[v] * (b->desc[v].model == AKMC_EAM ? 4.0 : 1.0) *
                      (1.0 + 0.05 * b->desc[v].n_vac);
        work[v] = {-cost, v};
    }
    std::stable_sort(work.begin(), work.end());   // largest expected work first
    for (int32_t v = 0; v < b->n; ++v) order[v] = work[v].second;
    AKMC_CUDA(cudaMemcpyAsync(b->base + b->lo.targets, stg, (sizeof(uint64_t) + sizeof(int32_t)) * b->n,
                              cudaMemcpyHostToDevice, s));
    AKMC_CUDA(cudaEventRecord(b->staging_done[slot], s));
    b->staging_used[slot] = true;
    if (b->occupancy[b->warps] == 0) b->occupancy[b->warps] = step_occupancy(b->warps, b->lo.max_nv, b->lo.max_P, b->lo.win);
    return AKMC_OK;
}

akmc_status akmc_launch_step(akmc_batch* b, akmc_stream stream) {
    if (!b) return fail(AKMC_EINVAL, "batch is NULL");
    if (b->dirty) return fail(AKMC_EINVAL, "rates are out of date after a state load: call akmc_compute_rates");
    cudaStream_t s = (cudaStream_t)stream;
    if (b->occupancy[b->warps] == 0) b->occupancy[b->warps] = step_occupancy(b->warps, b->lo.max_nv, b->lo.max_P, b->lo.win);
    AKMC_CUDA(cudaMemsetAsync(b->base + b->lo.queue, 0, sizeof(uint32_t), s));
    int per_sm = b->ctas_per_sm > 0 ? b->ctas_per_sm : b->occupancy[b->warps];
    if (per_sm < 1) per_sm = 1;
    int grid = std::min<long long>((long long)per_sm * b->n_sm, b->n);
    cudaError_t e = launch_step(b->args(), b->warps, grid, s);
    if (e != cudaSuccess) return fail(AKMC_ECUDA, "step kernel: %s", cudaGetErrorString(e));
    return AKMC_OK;
}

akmc_status akmc_step_n(akmc_batch* b, const uint64_t* n_events, akmc_stream stream) {
    if (!b || !n_events) return fail(AKMC_EINVAL, "batch or n_events is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (b->dirty) {
        akmc_status st = rebuild(b, s);
        if (st != AKMC_OK) return st;
    }
    akmc_status st = akmc_set_targets(b, n_events, stream);
    if (st != AKMC_OK) return st;
    return akmc_launch_step(b, stream);
}

namespace {
akmc_status sl_check(akmc_batch* b, int32_t voxel, int32_t Sc, double window_s) {
    if (!b) return fail(AKMC_EINVAL, "batch is NULL");
    if (voxel < 0 || voxel >= b->n) return fail(AKMC_EINVAL, "voxel %d out of range", voxel);
    const int L = b->desc[voxel].L;
    if (Sc < 8 || Sc % 2 || L % Sc)
        return fail(AKMC_EINVAL, "sector_cells %d must be even, >= 8 and divide L = %d", Sc, L);
    if (!(window_s > 0.0) || !std::isfinite(window_s)) return fail(AKMC_EINVAL, "window must be positive and finite");
    return AKMC_OK;
}
}  // namespace

namespace {
// Both sublattice forms.  skip_sector >= 0 only with the asynchronous form (test hook).
akmc_status sl_run(akmc_batch* b, int32_t voxel, uint64_t superstep0, uint32_t n_supersteps, int32_t Sc,
                   double window_s, bool asynchronous, int skip_sector, cudaStream_t s) {
    akmc_status st = sl_check(b, voxel, Sc, window_s);
    if (st != AKMC_OK) return st;
    if (n_supersteps == 0) return AKMC_OK;
    if (b->dirty) {
        st = rebuild(b, s);
        if (st != AKMC_OK) return st;
    }
    const BatchArgs a = b->args();
    const int ns = b->desc[voxel].L / Sc, n_sec = ns * ns * ns;
    int32_t* words = (int32_t*)(b->base + b->lo.sl_done);
    int32_t* stale = words + 4 + b->lo.sl_max_sectors;
    // stored rates are current here (kept by the step kernel, rebuilt after a load)
    AKMC_CUDA(cudaMemsetAsync(words, 0, sizeof(int32_t) * (4 + (size_t)b->lo.sl_max_sectors + b->desc[voxel].n_vac), s));
    cudaError_t e;
    if (asynchronous) {
        int grid = 0;
        e = launch_sublattice_async(a, voxel, (uint32_t)superstep0, n_supersteps, Sc, n_sec, window_s, words + 4,
                                    words, stale, skip_sector, b->n_sm, &grid, s);
        if (e != cudaSuccess) return fail(AKMC_ECUDA, "asynchronous sublattice kernel: %s", cudaGetErrorString(e));
    } else {
        e = sl_prepare(a);
        if (e != cudaSuccess) return fail(AKMC_ECUDA, "sublattice kernel attribute: %s", cudaGetErrorString(e));
        for (uint32_t i = 0; i < n_supersteps; ++i) {
            e = launch_sublattice(a, voxel, (uint32_t)(superstep0 + i), Sc, n_sec, window_s, stale, s);
            if (e != cudaSuccess) return fail(AKMC_ECUDA, "sublattice kernel: %s", cudaGetErrorString(e));
        }
    }
    // the supersteps keep lattice, densities, positions, clock and counter; the
    // voxel's rates and tree are rebuilt from the new lattice
    e = launch_rebuild(a, 8, (const int32_t*)(b->base + b->lo.ident) + voxel, 1, s);
    if (e != cudaSuccess) return fail(AKMC_ECUDA, "rebuild kernel: %s", cudaGetErrorString(e));
    return AKMC_OK;
}
}  // namespace

akmc_status akmc_step_sublattice_async(akmc_batch* b, int32_t voxel, uint64_t superstep0, uint32_t n_supersteps,
                                       int32_t sector_cells, double window_s, akmc_stream stream) {
    return sl_run(b, voxel, superstep0, n_supersteps, sector_cells, window_s, true, -1, (cudaStream_t)stream);
}

akmc_status akmc_step_sublattice(akmc_batch* b, int32_t voxel, uint64_t superstep0, uint32_t n_supersteps,
                                 int32_t sector_cells, double window_s, akmc_stream stream) {
    return sl_run(b, voxel, superstep0, n_supersteps, sector_cells, window_s, false, -1, (cudaStream_t)stream);
}

akmc_status akmc_test_sublattice_stall(akmc_batch* b, int32_t voxel, uint32_t n_supersteps, int32_t sector_cells,
                                       double window_s, int32_t stall_sector, akmc_stream stream) {
    if (b && voxel >= 0 && voxel < b->n && sector_cells > 0) {
        const int ns = b->desc[voxel].L / sector_cells;
        if (stall_sector < 0 || stall_sector >= ns * ns * ns)
            return fail(AKMC_EINVAL, "stall_sector %d out of range", stall_sector);
    }
    return sl_run(b, voxel, 0, n_supersteps, sector_cells, window_s, true, stall_sector, (cudaStream_t)stream);
}

akmc_status akmc_reset_voxels(akmc_batch* b, const int32_t* slots, const akmc_voxel_desc* descs, int32_t n,
                              akmc_stream stream) {
    if (!b || (n > 0 && (!slots || !descs))) return fail(AKMC_EINVAL, "NULL argument");
    if (n < 0 || n > b->n) return fail(AKMC_EINVAL, "bad slot count %d", n);
    if (n == 0) return AKMC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<char> seen(b->n, 0);
    for (int32_t i = 0; i < n; ++i) {
        const int32_t v = slots[i];
        if (v < 0 || v >= b->n || seen[v]) return fail(AKMC_EINVAL, "slot %d out of range or repeated", v);
        seen[v] = 1;
        const akmc_voxel_desc& d = descs[i];
        const akmc_voxel_desc& o = b->desc[v];
        if (d.L != o.L || d.n_vac != o.n_vac || d.model != o.model)
            return fail(AKMC_EINVAL, "slot %d: a new voxel must keep L, n_vac and model", v);
        if (d.precision != AKMC_FP64 && d.precision != AKMC_SPLIT)
            return fail(AKMC_EINVAL, "slot %d: bad precision", v);
        if (!(d.T > 0.0) || !std::isfinite(d.T)) return fail(AKMC_EINVAL, "slot %d: bad T", v);
        int32_t cnt[4];
        for (int k = 0; k < 3; ++k)
            if (!(d.frac[k] >= 0.0) || !(d.frac[k] <= 1.0)) return fail(AKMC_EINVAL, "slot %d: bad frac", v);
        species_counts(d, cnt);
        if ((long long)cnt[0] + cnt[1] + cnt[2] + cnt[3] > 2LL * d.L * d.L * d.L)
            return fail(AKMC_EINVAL, "slot %d: more solutes than sites", v);
    }
    const Layout& lo = b->lo;
    std::vector<int4> items, strips;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t v = slots[i];
        const akmc_voxel_desc& d = descs[i];
        b->desc[v] = d;
        VoxelDev& V = b->vox_host[v];
        V.status = AKMC_OK;
        V.precision = d.precision;
        species_counts(d, V.counts);
        V.beta = 1.0 / (kKB * d.T);
        for (int k = 0; k < 3; ++k) V.frac[k] = d.frac[k];
        V.T = d.T;
        V.seed = d.seed;
        V.uid = d.uid;
        V.n_events = 0;
        V.t_hi = V.t_lo = 0.0;
        V.etab_ok = 0;
        AKMC_CUDA(cudaMemcpyAsync(b->base + lo.vox + sizeof(VoxelDev) * v, &V, sizeof V, cudaMemcpyHostToDevice, s));
        AKMC_CUDA(cudaMemsetAsync(V.species, 0, V.N, s));
        AKMC_CUDA(cudaMemsetAsync(V.vac_pos, 0, 4 * (size_t)V.nv, s));
        AKMC_CUDA(cudaMemsetAsync(V.vac_disp, 0, 12 * (size_t)V.nv, s));
        AKMC_CUDA(cudaMemsetAsync(V.rates, 0, 64 * (size_t)V.nv, s));
        AKMC_CUDA(cudaMemsetAsync(V.dE, 0, 64 * (size_t)V.nv, s));
        AKMC_CUDA(cudaMemsetAsync(V.hop_sp, 0, 8 * (size_t)V.nv, s));
        AKMC_CUDA(cudaMemsetAsync(V.tree, 0, 16 * (size_t)V.P, s));
        if (V.log) AKMC_CUDA(cudaMemsetAsync(V.log, 0, 4 * (size_t)V.log_cap, s));
        for (const int4& it : lo.item_list)
            if (it.x == v) items.push_back(it);
        for (const int4& it : lo.strip_list)
            if (it.x == v) strips.push_back(it);
    }
    int32_t* list = (int32_t*)(b->base + lo.reset_list);
    AKMC_CUDA(cudaMemcpyAsync(list, slots, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    VoxelDev* vox = (VoxelDev*)(b->base + lo.vox);
    launch_place(vox, n, list, s);
    AKMC_CUDA(cudaGetLastError());
    AKMC_CUDA(launch_rate_tables(vox, n, (const ModelDev*)(b->base + lo.model), list, s));
    BatchArgs a = b->args();
    if (!items.empty())
        AKMC_CUDA(cudaMemcpyAsync(b->base + lo.reset_items, items.data(), sizeof(int4) * items.size(),
                                  cudaMemcpyHostToDevice, s));
    if (!strips.empty())
        AKMC_CUDA(cudaMemcpyAsync(b->base + lo.reset_strips, strips.data(), sizeof(int4) * strips.size(),
                                  cudaMemcpyHostToDevice, s));
    if (!items.empty() || !strips.empty())
        AKMC_CUDA(launch_density(a.vox, a.model, a.tab, (const int4*)(b->base + lo.reset_items), (int)items.size(),
                                 (const int4*)(b->base + lo.reset_strips), (int)strips.size(), lo.strip_dyn, s));
    AKMC_CUDA(launch_rebuild(a, 8, list, n, s));
    // pageable sources above are staged by the copies; the tile list must outlive its copy
    AKMC_CUDA(cudaStreamSynchronize(s));
    return AKMC_OK;
}

akmc_status akmc_read_state(akmc_batch* b, int32_t voxel, akmc_state* out, akmc_stream stream) {
    if (!b || !out) return fail(AKMC_EINVAL, "batch or out is NULL");
    if (voxel < 0 || voxel >= b->n) return fail(AKMC_EINVAL, "voxel %d out of range", voxel);
    cudaStream_t s = (cudaStream_t)stream;
    const VoxelDev& H = b->vox_host[voxel];
    VoxelDev cur;
    AKMC_CUDA(cudaMemcpyAsync(&cur, b->base + b->lo.vox + sizeof(VoxelDev) * voxel, sizeof cur,
                              cudaMemcpyDeviceToHost, s));
    if (out->species) AKMC_CUDA(cudaMemcpyAsync(out->species, H.species, H.N, cudaMemcpyDeviceToHost, s));
    if (out->vac_pos)
        AKMC_CUDA(cudaMemcpyAsync(out->vac_pos, H.vac_pos, 4 * (size_t)H.nv, cudaMemcpyDeviceToHost, s));
    if (out->vac_disp)
        AKMC_CUDA(cudaMemcpyAsync(out->vac_disp, H.vac_disp, 12 * (size_t)H.nv, cudaMemcpyDeviceToHost, s));
    if (out->rates)
        AKMC_CUDA(cudaMemcpyAsync(out->rates, H.rates, 64 * (size_t)H.nv, cudaMemcpyDeviceToHost, s));
    if (out->dE) AKMC_CUDA(cudaMemcpyAsync(out->dE, H.dE, 64 * (size_t)H.nv, cudaMemcpyDeviceToHost, s));
    if (out->event_log && b->log_cap > 0)
        AKMC_CUDA(cudaMemcpyAsync(out->event_log, H.log, 4 * (size_t)b->log_cap, cudaMemcpyDeviceToHost, s));
    AKMC_CUDA(cudaStreamSynchronize(s));
    out->t_hi = cur.t_hi;
    out->t_lo = cur.t_lo;
    out->n_events = cur.n_events;
    out->status = cur.status;
    out->L = H.L;
    out->n_vac = H.nv;
    return AKMC_OK;
}

akmc_status akmc_read_density(akmc_batch* b, int32_t voxel, int32_t* host_rho, akmc_stream stream) {
    if (!b || !host_rho) return fail(AKMC_EINVAL, "batch or host_rho is NULL");
    if (voxel < 0 || voxel >= b->n) return fail(AKMC_EINVAL, "voxel %d out of range", voxel);
    const VoxelDev& H = b->vox_host[voxel];
    if (!H.rho) return fail(AKMC_EINVAL, "voxel %d uses the pair model (no densities)", voxel);
    if (b->dirty) return fail(AKMC_EINVAL, "densities are out of date after a state load; call akmc_compute_rates");
    cudaStream_t s = (cudaStream_t)stream;
    AKMC_CUDA(cudaMemcpyAsync(host_rho, H.rho, sizeof(int32_t) * (size_t)H.N, cudaMemcpyDeviceToHost, s));
    AKMC_CUDA(cudaStreamSynchronize(s));
    return AKMC_OK;
}

akmc_status akmc_load_state(akmc_batch* b, int32_t voxel, const uint8_t* species, const int32_t* vac_pos,
                            double t_hi, double t_lo, uint64_t n_events, akmc_stream stream) {
    if (!b || !species || !vac_pos) return fail(AKMC_EINVAL, "NULL argument");
    if (voxel < 0 || voxel >= b->n) return fail(AKMC_EINVAL, "voxel %d out of range", voxel);
    cudaStream_t s = (cudaStream_t)stream;
    const VoxelDev& V = b->vox_host[voxel];
    int nvac = 0;
    for (int i = 0; i < V.N; ++i) {
        if (species[i] > kVac) return fail(AKMC_EINVAL, "species code %d at site %d", species[i], i);
        nvac += species[i] == kVac;
    }
    if (nvac != V.nv) return fail(AKMC_EINVAL, "lattice has %d vacancies, voxel has %d slots", nvac, V.nv);
    for (int q = 0; q < V.nv; ++q)
        if (vac_pos[q] < 0 || vac_pos[q] >= V.N || species[vac_pos[q]] != kVac)
            return fail(AKMC_EINVAL, "vac_pos[%d] is not a vacancy site", q);
    if (!std::isfinite(t_hi) || !std::isfinite(t_lo)) return fail(AKMC_EINVAL, "clock must be finite");
    AKMC_CUDA(cudaStreamSynchronize(s));
    double* io = (double*)(b->base + b->lo.io);
    const double clk[2] = {t_hi, t_lo};
    AKMC_CUDA(cudaMemcpyAsync(V.species, species, V.N, cudaMemcpyHostToDevice, s));
    AKMC_CUDA(cudaMemcpyAsync(V.vac_pos, vac_pos, 4 * (size_t)V.nv, cudaMemcpyHostToDevice, s));
    AKMC_CUDA(cudaMemcpyAsync(io, clk, sizeof clk, cudaMemcpyHostToDevice, s));
    AKMC_CUDA(cudaMemcpyAsync(io + 2, &n_events, sizeof n_events, cudaMemcpyHostToDevice, s));
    AKMC_CUDA(launch_voxel_load((VoxelDev*)(b->base + b->lo.vox) + voxel, io, s));
    AKMC_CUDA(cudaStreamSynchronize(s));
    b->dirty = true;
    return AKMC_OK;
}

akmc_status akmc_load_batch_state(akmc_batch* b, const uint8_t* species, const int32_t* vac_pos,
                                  const double* t_hi, const double* t_lo, const uint64_t* n_events,
                                  akmc_stream stream) {
    if (!b || !species || !vac_pos) return fail(AKMC_EINVAL, "NULL argument");
    if ((t_hi == nullptr) != (t_lo == nullptr)) return fail(AKMC_EINVAL, "give both t_hi and t_lo or neither");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = b->n;
    double* io = (double*)(b->base + b->lo.io);
    AKMC_CUDA(cudaMemcpyAsync(b->base + b->lo.b_species, species, b->lo.tot_N, cudaMemcpyHostToDevice, s));
    AKMC_CUDA(cudaMemcpyAsync(b->base + b->lo.b_pos, vac_pos, sizeof(int32_t) * b->lo.tot_nv,
                              cudaMemcpyHostToDevice, s));
    if (t_hi) {
        AKMC_CUDA(cudaMemcpyAsync(io, t_hi, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        AKMC_CUDA(cudaMemcpyAsync(io + n, t_lo, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    }
    if (n_events)
        AKMC_CUDA(cudaMemcpyAsync(io + 2 * n, n_events, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, s));
    AKMC_CUDA(launch_batch_load((VoxelDev*)(b->base + b->lo.vox), io, n, t_hi != nullptr, n_events != nullptr, s));
    b->dirty = true;
    return AKMC_OK;
}

akmc_status akmc_read_batch_state(akmc_batch* b, uint8_t* species, int32_t* vac_pos, int32_t* vac_disp,
                                  double* t_hi, double* t_lo, uint64_t* n_events, int32_t* status,
                                  akmc_stream stream) {
    if (!b) return fail(AKMC_EINVAL, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = b->n;
    double* io = (double*)(b->base + b->lo.io);
    if (species)
        AKMC_CUDA(cudaMemcpyAsync(species, b->base + b->lo.b_species, b->lo.tot_N, cudaMemcpyDeviceToHost, s));
    if (vac_pos)
        AKMC_CUDA(cudaMemcpyAsync(vac_pos, b->base + b->lo.b_pos, sizeof(int32_t) * b->lo.tot_nv,
                                  cudaMemcpyDeviceToHost, s));
    if (vac_disp)
        AKMC_CUDA(cudaMemcpyAsync(vac_disp, b->base + b->lo.b_disp, sizeof(int32_t) * 3 * b->lo.tot_nv,
                                  cudaMemcpyDeviceToHost, s));
    if (t_hi || t_lo || n_events || status) {
        AKMC_CUDA(launch_batch_read((const VoxelDev*)(b->base + b->lo.vox), io, n, s));
        if (t_hi) AKMC_CUDA(cudaMemcpyAsync(t_hi, io, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        if (t_lo) AKMC_CUDA(cudaMemcpyAsync(t_lo, io + n, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        if (n_events)
            AKMC_CUDA(cudaMemcpyAsync(n_events, io + 2 * n, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, s));
        if (status)
            AKMC_CUDA(cudaMemcpyAsync(status, io + 3 * n, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    }
    return AKMC_OK;
}

akmc_status akmc_workload_proxy(akmc_batch* b, double* W, double* M_hat, double* E_hat, akmc_stream stream) {
    if (!b) return fail(AKMC_EINVAL, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (b->dirty) {
        akmc_status st = rebuild(b, s);
        if (st != AKMC_OK) return st;
    }
    const int n = b->n;
    double* io = (double*)(b->base + b->lo.io);
    AKMC_CUDA(launch_proxy((const VoxelDev*)(b->base + b->lo.vox), (const ModelDev*)(b->base + b->lo.model), io, n, s));
    std::vector<double> h(3 * (size_t)n);
    AKMC_CUDA(cudaMemcpyAsync(h.data(), io, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    AKMC_CUDA(cudaStreamSynchronize(s));
    for (int v = 0; v < n; ++v) {
        if (W) W[v] = h[v];
        if (M_hat) M_hat[v] = h[n + v];
        if (E_hat) E_hat[v] = h[2 * (size_t)n + v];
    }
    return AKMC_OK;
}

size_t akmc_batch_sites(const akmc_batch* b) { return b ? b->lo.tot_N : 0; }
int64_t akmc_batch_vacancies(const akmc_batch* b) { return b ? (int64_t)b->lo.tot_nv : 0; }

akmc_status akmc_sync_status(akmc_batch* b, akmc_stream stream, int32_t* per_voxel) {
    if (!b) return fail(AKMC_EINVAL, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<VoxelDev> cur(b->n);
    int32_t bst = 0;
    AKMC_CUDA(cudaMemcpyAsync(cur.data(), b->base + b->lo.vox, sizeof(VoxelDev) * b->n,
                              cudaMemcpyDeviceToHost, s));
    AKMC_CUDA(cudaMemcpyAsync(&bst, b->base + b->lo.status, sizeof bst, cudaMemcpyDeviceToHost, s));
    AKMC_CUDA(cudaStreamSynchronize(s));
    AKMC_CUDA(cudaGetLastError());
    if (bst != 0) return fail((akmc_status)bst, "model setup rejected the tables (status %d)", bst);
    akmc_status first = AKMC_OK;
    for (int32_t v = 0; v < b->n; ++v) {
        if (per_voxel) per_voxel[v] = cur[v].status;
        if (first == AKMC_OK && cur[v].status != AKMC_OK) first = (akmc_status)cur[v].status;
    }
    return first;
}

akmc_status akmc_cluster_hist(akmc_batch* b, int32_t voxel, int32_t mode, int64_t hist[8], akmc_stream stream) {
    if (!b || !hist) return fail(AKMC_EINVAL, "NULL argument");
    if (voxel < 0 || voxel >= b->n) return fail(AKMC_EINVAL, "voxel %d out of range", voxel);
    if (mode != 0 && mode != 1) return fail(AKMC_EINVAL, "mode must be 0 or 1");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* dh = (unsigned long long*)(b->base + b->lo.hist);
    cudaError_t e = launch_cluster(b->vox_host.data(), voxel, b->vox_host[voxel].N,
                                   (const Tables*)(b->base + b->lo.tab), mode,
                                   (int32_t*)(b->base + b->lo.labels), (int32_t*)(b->base + b->lo.sizes), dh, s);
    if (e != cudaSuccess) return fail(AKMC_ECUDA, "cluster kernels: %s", cudaGetErrorString(e));
    unsigned long long h[8];
    AKMC_CUDA(cudaMemcpyAsync(h, dh, sizeof h, cudaMemcpyDeviceToHost, s));
    AKMC_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < 8; ++i) hist[i] = (int64_t)h[i];
    return AKMC_OK;
}

akmc_status akmc_set_launch(akmc_batch* b, int32_t warps, int32_t ctas_per_sm) {
    if (!b) return fail(AKMC_EINVAL, "batch is NULL");
    if (warps != 1 && warps != 2 && warps != 4 && warps != 8 && warps != 16)
        return fail(AKMC_EINVAL, "warps must be 1, 2, 4, 8 or 16");
    if (ctas_per_sm < 0 || ctas_per_sm > 64) return fail(AKMC_EINVAL, "ctas_per_sm out of range");
    b->warps = warps;
    b->ctas_per_sm = ctas_per_sm;
    return AKMC_OK;
}

int32_t akmc_n_voxels(const akmc_batch* b) { return b ? b->n : 0; }

void akmc_destroy_batch(akmc_batch* b) {
    if (!b) return;
    for (int i = 0; i < akmc_batch::kStage; ++i)
        if (b->staging_done[i]) {
            cudaEventSynchronize(b->staging_done[i]);
            cudaEventDestroy(b->staging_done[i]);
        }
    if (b->staging) cudaFreeHost(b->staging);
    delete b;
}

}  // extern "C"
