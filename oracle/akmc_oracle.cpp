// akmc_oracle.cpp -- TEST INFRASTRUCTURE ONLY (see akmc_oracle.h).
//
// Plain serial float64 rejection-free vacancy AKMC on a periodic bcc lattice.
// Every quantity is computed from its definition with plain loops; there is no
// blocking, fusion or reordering beyond the algorithm's own steps:
//   (a1) lattice + vacancy slots   (a2/a3) hop energy change   (a4) barrier and rate
//   (a5) rate sums in a binary tree (a6) selection              (a7) swap (+ density update)
//   (a8) refresh of affected rates  (a9) compensated clock
// Paper passages: every migration direction of every vacancy is enumerated and
// rated (Sec. "Compute-Centric Reformulation"); the time step is inversely
// proportional to the total rate (Sec. "Current State of the Art"); rates are
// Arrhenius (Eq. 8); inadmissible transitions are masked out and all events
// compete globally (Eq. 1-2); voxels are periodic and independent
// (Sec. "Mesoscopic Voxel-Parallel Formulation").  The synchronous sublattice
// schedule (orc_step_sublattice; Sec. "Asynchronous Sublattice Parallelism"
// names its synchronous form and the readiness refinement) runs the sectors of
// each superstep one after another; it is pinned by sector-order independence,
// conservation, the clock and the pure-Fe scheduled walk (test_oracle_sublattice).
#include "akmc_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

constexpr int FE = 0, VAC = 4;
constexpr double KB = 8.617333262e-5;        // eV/K, CODATA 2018
constexpr int RHO_BITS = 24;                  // fixed-point density unit 2^-24

struct Off { int dx, dy, dz, shell; };

// Squared half-unit length -> bcc shell number (0: not within the cutoff).
int shell_of_len2(int l2) {
    switch (l2) {
        case 3: return 1;    // (1,1,1)   a*sqrt(3)/2
        case 4: return 2;    // (2,0,0)   a
        case 8: return 3;    // (2,2,0)   a*sqrt(2)
        case 11: return 4;   // (3,1,1)   a*sqrt(11)/2
        case 12: return 5;   // (2,2,2)   a*sqrt(3)
        default: return 0;
    }
}
const int SHELL_LEN2[6] = {0, 3, 4, 8, 11, 12};

struct Shells {
    std::vector<Off> n12;   // 1nn then 2nn (pair model)
    std::vector<Off> sph;   // shells 1..5 within 5.6 A (EAM), 58 offsets
    Shells() {
        for (int want = 1; want <= 5; ++want)
            for (int dz = -4; dz <= 4; ++dz)
                for (int dy = -4; dy <= 4; ++dy)
                    for (int dx = -4; dx <= 4; ++dx) {
                        bool odd = (dx & 1) && (dy & 1) && (dz & 1);
                        bool even = !(dx & 1) && !(dy & 1) && !(dz & 1);
                        if (!(odd || even)) continue;
                        int s = shell_of_len2(dx * dx + dy * dy + dz * dz);
                        if (s != want) continue;
                        Off o{dx, dy, dz, s};
                        sph.push_back(o);
                        if (s <= 2) n12.push_back(o);
                    }
    }
};
const Shells& shells() { static Shells s; return s; }

// 1nn hop direction: dir = (dx<0) + 2(dy<0) + 4(dz<0).
void dirvec(int dir, int& dx, int& dy, int& dz) {
    dx = (dir & 1) ? -1 : 1;
    dy = (dir & 2) ? -1 : 1;
    dz = (dir & 4) ? -1 : 1;
}

uint32_t mulhi32(uint32_t a, uint32_t b, uint32_t* lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *lo = (uint32_t)p;
    return (uint32_t)(p >> 32);
}

int pair_index(int a, int b) {
    if (a > b) std::swap(a, b);
    return a * (7 - a) / 2 + b;
}

// Cubic Hermite interpolation on a uniform grid from (value, derivative) pairs.
double hermite(const double* tab, int k, double t, double h) {
    double v0 = tab[2 * k], d0 = tab[2 * k + 1] * h;
    double v1 = tab[2 * k + 2], d1 = tab[2 * k + 3] * h;
    double t2 = t * t, t3 = t2 * t;
    double h00 = 2.0 * t3 - 3.0 * t2 + 1.0;
    double h10 = t3 - 2.0 * t2 + t;
    double h01 = -2.0 * t3 + 3.0 * t2;
    double h11 = t3 - t2;
    return h00 * v0 + h10 * d0 + h01 * v1 + h11 * d1;
}

double table_at_r(const double* tab, int n, double r_cut, double r) {
    double dr = r_cut / (double)(n - 1);
    double x = r / dr;
    int k = (int)std::floor(x);
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    return hermite(tab, k, x - (double)k, dr);
}

int rho_shift(double rho_h) {
    // rho_h = 2^-e with 0 <= e <= 24  ->  knot spacing in fixed units = 2^(24-e)
    int e = 0;
    double h = rho_h;
    while (h < 1.0 && e <= RHO_BITS) { h *= 2.0; ++e; }
    if (h != 1.0 || e > RHO_BITS) return -1;
    return RHO_BITS - e;
}

}  // namespace

struct orc_voxel {
    int L = 0, N = 0, nv = 0, model = 0;
    double T = 0, beta = 0;
    uint64_t seed = 0, uid = 0;
    // model
    double eps1[25], eps2[25], E0[4], nu = 0, a = 0;
    int n_rho = 0, shift = 0;
    double rho_h = 0;
    std::vector<double> F_tab;
    double phi_s[10][6];
    int64_t fq[4][6];
    // state
    std::vector<uint8_t> sp;
    std::vector<int64_t> rho;
    std::vector<int> pos, disp;
    std::vector<double> rate, dE;
    int P = 1;
    std::vector<double> tree;
    double t_hi = 0, t_lo = 0;
    uint64_t n = 0;
    int status = ORC_OK;
    double sl_T = 0;
    mutable int numeric = 0;
    // debug
    int debug = 0;
    uint64_t cnt[5] = {0, 0, 0, 0, 0};
    std::vector<int> tdisp;
    std::vector<uint32_t> stamp;
    uint32_t epoch = 0;
};

namespace {

int site_of(const orc_voxel* v, int X, int Y, int Z) {
    int M = 2 * v->L;
    X = ((X % M) + M) % M;
    Y = ((Y % M) + M) % M;
    Z = ((Z % M) + M) % M;
    int b = X & 1;
    return ((((Z >> 1) * v->L + (Y >> 1)) * v->L + (X >> 1)) << 1) | b;
}

void coords_of(const orc_voxel* v, int s, int& X, int& Y, int& Z) {
    int b = s & 1, c = s >> 1;
    int x = c % v->L, y = (c / v->L) % v->L, z = c / (v->L * v->L);
    X = 2 * x + b;
    Y = 2 * y + b;
    Z = 2 * z + b;
}

int nbr(const orc_voxel* v, int s, int dx, int dy, int dz) {
    int X, Y, Z;
    coords_of(v, s, X, Y, Z);
    return site_of(v, X + dx, Y + dy, Z + dz);
}

int hop_target(const orc_voxel* v, int w, int dir) {
    int dx, dy, dz;
    dirvec(dir, dx, dy, dz);
    return nbr(v, w, dx, dy, dz);
}

double eps(const orc_voxel* v, int shell, int a, int b) {
    return shell == 1 ? v->eps1[a * 5 + b] : v->eps2[a * 5 + b];
}

double phi(const orc_voxel* v, int a, int b, int shell) {
    return v->phi_s[pair_index(a, b)][shell];
}

// F_a at a fixed-point density; the knot spacing is a power of two so the
// interval index and the local coordinate are exact.  Densities outside the
// table are clamped to the end interval and flagged.
double embed(const orc_voxel* v, int a, int64_t rho_fixed) {
    int64_t k = rho_fixed >> v->shift;
    int64_t last = (int64_t)v->n_rho - 1;
    if (rho_fixed < 0 || rho_fixed > (last << v->shift)) v->numeric = 1;
    if (k > last - 1) k = last - 1;
    if (k < 0) k = 0;
    double t = (double)(rho_fixed - (k << v->shift)) / (double)((int64_t)1 << v->shift);
    return hermite(&v->F_tab[(size_t)a * v->n_rho * 2], (int)k, t, v->rho_h);
}

// ---- (a2) pair model hop energy change, local form --------------------------
// Vacancy at w exchanges with atom A at the 1nn site m.  Only bonds of w and
// m change: every neighbour j of w (except m) trades eps(V,s_j) for eps(A,s_j),
// every neighbour j of m (except w) trades eps(A,s_j) for eps(V,s_j).
double de_pair_local(const orc_voxel* v, const uint8_t* sp, int w, int m) {
    const Shells& S = shells();
    int A = sp[m];
    double de = 0.0;
    for (const Off& o : S.n12) {
        int j = nbr(v, w, o.dx, o.dy, o.dz);
        if (j == m) continue;
        de += eps(v, o.shell, A, sp[j]) - eps(v, o.shell, VAC, sp[j]);
    }
    for (const Off& o : S.n12) {
        int j = nbr(v, m, o.dx, o.dy, o.dz);
        if (j == w) continue;
        de += eps(v, o.shell, VAC, sp[j]) - eps(v, o.shell, A, sp[j]);
    }
    return de;
}

// Full-lattice pair energy E = 1/2 sum_i sum_{j in N1(i)} eps1 + 1/2 sum_i sum_{j in N2(i)} eps2
// (the vacancy is a species with its own rows).
double energy_pair(const orc_voxel* v, const uint8_t* sp) {
    const Shells& S = shells();
    double E = 0.0;
    for (int i = 0; i < v->N; ++i)
        for (const Off& o : S.n12) {
            int j = nbr(v, i, o.dx, o.dy, o.dz);
            E += 0.5 * eps(v, o.shell, sp[i], sp[j]);
        }
    return E;
}

// ---- EAM: rho_i = sum_{j in S(i), s_j != V} f_{s_j}(r_ij) (fixed point) ------
int64_t rho_scratch(const orc_voxel* v, const uint8_t* sp, int i) {
    const Shells& S = shells();
    int64_t r = 0;
    for (const Off& o : S.sph) {
        int j = nbr(v, i, o.dx, o.dy, o.dz);
        if (sp[j] != VAC) r += v->fq[sp[j]][o.shell];
    }
    return r;
}

// Energy of site i: F_{s_i}(rho_i) + 1/2 sum_{j in S(i), s_j != V} phi_{s_i s_j}(r_ij).
double site_energy_eam(const orc_voxel* v, const uint8_t* sp, int i) {
    if (sp[i] == VAC) return 0.0;
    const Shells& S = shells();
    double e = embed(v, sp[i], rho_scratch(v, sp, i));
    for (const Off& o : S.sph) {
        int j = nbr(v, i, o.dx, o.dy, o.dz);
        if (sp[j] != VAC) e += 0.5 * phi(v, sp[i], sp[j], o.shell);
    }
    return e;
}

double energy_eam(const orc_voxel* v, const uint8_t* sp) {
    double E = 0.0;
    for (int i = 0; i < v->N; ++i) E += site_energy_eam(v, sp, i);
    return E;
}

// ---- (a3) EAM hop energy change, local form ------------------------------
// Atom A moves m -> w.  Densities change only on S(w) and S(m):
//   drho_i = f_A(r_iw)[i in S(w)] - f_A(r_im)[i in S(m)].
// dE = sum_{i in S(w)uS(m), i != w,m, s_i != V} [F_{s_i}(rho_i + drho_i) - F_{s_i}(rho_i)]
//    + F_A(rho_w - f_A(r_wm)) - F_A(rho_m)
//    + sum_{j in S(w), j != m, s_j != V} phi_{A s_j}(r_wj) - sum_{j in S(m), j != w, s_j != V} phi_{A s_j}(r_mj)
double de_eam_local(const orc_voxel* v, const uint8_t* sp, const int64_t* rho, int w, int m) {
    const Shells& S = shells();
    int A = sp[m];
    std::vector<int> aff;
    std::vector<int64_t> drho;
    auto add = [&](int i, int64_t d) {
        for (size_t q = 0; q < aff.size(); ++q)
            if (aff[q] == i) { drho[q] += d; return; }
        aff.push_back(i);
        drho.push_back(d);
    };
    int64_t f_wm = 0;
    for (const Off& o : S.sph) {
        int i = nbr(v, w, o.dx, o.dy, o.dz);
        if (i == m) f_wm += v->fq[A][o.shell];
        if (i == w || i == m) continue;
        add(i, v->fq[A][o.shell]);
    }
    for (const Off& o : S.sph) {
        int i = nbr(v, m, o.dx, o.dy, o.dz);
        if (i == w || i == m) continue;
        add(i, -v->fq[A][o.shell]);
    }
    double de = 0.0;
    for (size_t q = 0; q < aff.size(); ++q) {
        int i = aff[q];
        if (sp[i] == VAC) continue;
        de += embed(v, sp[i], rho[i] + drho[q]) - embed(v, sp[i], rho[i]);
    }
    de += embed(v, A, rho[w] - f_wm) - embed(v, A, rho[m]);
    for (const Off& o : S.sph) {
        int j = nbr(v, w, o.dx, o.dy, o.dz);
        if (j == m || sp[j] == VAC) continue;
        de += phi(v, A, sp[j], o.shell);
    }
    for (const Off& o : S.sph) {
        int j = nbr(v, m, o.dx, o.dy, o.dz);
        if (j == w || sp[j] == VAC) continue;
        de -= phi(v, A, sp[j], o.shell);
    }
    return de;
}

// ---- (a4) barrier and rate -------------------------------------------------
// Ea = max(0, dE, E0(A) + dE/2); rate = nu * exp(-Ea/(kB T)); a hop into a
// vacancy is not admissible (rate 0, the mask of Eq. 1).
double hop_rate_de(const orc_voxel* v, int slot, int dir, double* de_out) {
    int w = v->pos[slot];
    int m = hop_target(v, w, dir);
    int A = v->sp[m];
    if (A == VAC) {
        *de_out = 0.0;
        return 0.0;
    }
    double de = v->model == 0 ? de_pair_local(v, v->sp.data(), w, m)
                              : de_eam_local(v, v->sp.data(), v->rho.data(), w, m);
    *de_out = de;
    double Ea = std::max(std::max(0.0, de), v->E0[A] + 0.5 * de);
    return v->nu * std::exp(-(Ea * v->beta));
}

// ---- (a5) rate sums -----------------------------------------------------------
// Per vacancy S = ((g0+g1)+(g2+g3))+((g4+g5)+(g6+g7)); per voxel a complete
// binary tree over P = next_pow2(nv) vacancy sums, node = left + right.
double vacancy_sum(const double* g) {
    return ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]));
}

void tree_path_update(orc_voxel* v, int slot) {
    int i = (v->P + slot) >> 1;
    while (i >= 1) {
        v->tree[i] = v->tree[2 * i] + v->tree[2 * i + 1];
        i >>= 1;
    }
}

void refresh_vacancy(orc_voxel* v, int slot) {
    for (int d = 0; d < 8; ++d)
        v->rate[8 * slot + d] = hop_rate_de(v, slot, d, &v->dE[8 * slot + d]);
    v->tree[v->P + slot] = vacancy_sum(&v->rate[8 * slot]);
    tree_path_update(v, slot);
}

void rebuild_all(orc_voxel* v) {
    v->P = 1;
    while (v->P < v->nv) v->P <<= 1;
    v->tree.assign(2 * v->P, 0.0);
    v->rate.assign(8 * (size_t)v->nv, 0.0);
    v->dE.assign(8 * (size_t)v->nv, 0.0);
    if (v->model == 1) {
        v->rho.assign(v->N, 0);
        for (int i = 0; i < v->N; ++i) v->rho[i] = rho_scratch(v, v->sp.data(), i);
    }
    v->numeric = 0;
    for (int s = 0; s < v->nv; ++s) {
        for (int d = 0; d < 8; ++d)
            v->rate[8 * s + d] = hop_rate_de(v, s, d, &v->dE[8 * s + d]);
        v->tree[v->P + s] = vacancy_sum(&v->rate[8 * s]);
    }
    for (int i = v->P - 1; i >= 1; --i) v->tree[i] = v->tree[2 * i] + v->tree[2 * i + 1];
    if (v->numeric) v->status = ORC_ENUMERIC;
}

// ---- (a6) selection --------------------------------------------------------
// Descend with t: go left if t < left or the right subtree is empty, else
// subtract left and go right.  Lands on a nonzero leaf whenever the root is > 0.
int descend(const double* heap, int n_leaves, double& t) {
    int node = 1;
    while (node < n_leaves) {
        double l = heap[2 * node], r = heap[2 * node + 1];
        if (t < l || r == 0.0) {
            node = 2 * node;
        } else {
            t -= l;
            node = 2 * node + 1;
        }
    }
    return node - n_leaves;
}

void select_event(const orc_voxel* v, double t, int* slot, int* dir) {
    int s = descend(v->tree.data(), v->P, t);
    const double* g = &v->rate[8 * s];
    double h[16];
    for (int k = 0; k < 8; ++k) h[8 + k] = g[k];
    for (int i = 7; i >= 1; --i) h[i] = h[2 * i] + h[2 * i + 1];
    *slot = s;
    *dir = descend(h, 8, t);
}

// Plain cumulative scan over events e = 8*slot + dir (independent check).
// Also returns the distance from t to the nearest cumulative boundary.
int scan_select(const orc_voxel* v, double t, double* boundary_margin) {
    double c = 0.0, margin = INFINITY;
    int sel = -1, last_nz = -1;
    for (int e = 0; e < 8 * v->nv; ++e) {
        if (v->rate[e] > 0.0) last_nz = e;
        c += v->rate[e];
        margin = std::min(margin, std::fabs(t - c));
        if (sel < 0 && t < c) sel = e;
    }
    if (sel < 0) sel = last_nz;
    *boundary_margin = margin;
    return sel;
}

// ---- random numbers ----------------------------------------------------------
const uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;
const uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;

void philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PH_W0; k1 += PH_W1; }
        uint32_t lo0, lo1;
        uint32_t hi0 = mulhi32(PH_M0, c0, &lo0);
        uint32_t hi1 = mulhi32(PH_M1, c2, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void event_uniforms(uint64_t seed, uint64_t uid, uint64_t n, double* u1, double* u2) {
    uint32_t ctr[4] = {(uint32_t)n, (uint32_t)(n >> 32), (uint32_t)uid,
                       (uint32_t)(uid >> 32) & 0x7fffffffu};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    philox(ctr, key, x);
    uint64_t a = ((uint64_t)x[0] << 21) | (x[1] >> 11);
    uint64_t b = ((uint64_t)x[2] << 21) | (x[3] >> 11);
    *u1 = (double)a * 0x1p-53;          // [0, 1)
    *u2 = (double)(b + 1) * 0x1p-53;    // (0, 1]
}

// Placement draw k: a site uniform over [0, N) from 64 Philox bits (multiply-high).
int placement_draw(uint64_t seed, uint64_t uid, uint64_t k, int N) {
    uint32_t ctr[4] = {(uint32_t)k, (uint32_t)(k >> 32), (uint32_t)uid,
                       0x80000000u | (uint32_t)(uid >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    philox(ctr, key, x);
    uint64_t r = ((uint64_t)x[0] << 32) | x[1];
    return (int)(((unsigned __int128)r * (uint64_t)N) >> 64);
}

// ---- (a8) which vacancies does a hop w -> m affect? ------------------------------
// A vacancy at p reads species (and, for EAM, densities) on
//   pair: N12(p) u N12(m_k) for its 8 targets m_k;   EAM: {p} u S(p) u S(m_k).
// The hop changes species at {w, m} and (EAM) densities on {w,m} u S(w) u S(m).
bool affected(orc_voxel* v, int p, int w, int m) {
    const Shells& S = shells();
    const std::vector<Off>& shell = v->model == 0 ? S.n12 : S.sph;
    if (++v->epoch == 0) { std::fill(v->stamp.begin(), v->stamp.end(), 0u); v->epoch = 1; }
    uint32_t e = v->epoch;
    v->stamp[p] = e;
    for (const Off& o : shell) v->stamp[nbr(v, p, o.dx, o.dy, o.dz)] = e;
    for (int d = 0; d < 8; ++d) {
        int mk = hop_target(v, p, d);
        v->stamp[mk] = e;
        for (const Off& o : shell) v->stamp[nbr(v, mk, o.dx, o.dy, o.dz)] = e;
    }
    if (v->stamp[w] == e || v->stamp[m] == e) return true;
    if (v->model == 1) {
        for (const Off& o : S.sph) {
            if (v->stamp[nbr(v, w, o.dx, o.dy, o.dz)] == e) return true;
            if (v->stamp[nbr(v, m, o.dx, o.dy, o.dz)] == e) return true;
        }
    }
    return false;
}

void debug_checks(orc_voxel* v) {
    v->cnt[4]++;
    if ((v->debug & 4) && v->model == 1) {
        for (int i = 0; i < v->N; ++i)
            if (v->rho[i] != rho_scratch(v, v->sp.data(), i)) v->cnt[3]++;
    }
    if (v->debug & 1) {
        for (int s = 0; s < v->nv; ++s)
            for (int d = 0; d < 8; ++d) {
                double de;
                double r = hop_rate_de(v, s, d, &de);
                if (r != v->rate[8 * s + d]) v->cnt[0]++;
            }
        std::vector<double> t2(2 * v->P, 0.0);
        for (int s = 0; s < v->nv; ++s) t2[v->P + s] = vacancy_sum(&v->rate[8 * s]);
        for (int i = v->P - 1; i >= 1; --i) t2[i] = t2[2 * i] + t2[2 * i + 1];
        for (int i = 1; i < 2 * v->P; ++i)
            if (t2[i] != v->tree[i]) v->cnt[0]++;
    }
}

// One event: select, swap, clock, refresh.  Returns false if none could run.
bool one_event(orc_voxel* v, int32_t* log_entry, double* dt_entry) {
    double R = v->tree[1];
    if (!(R > 0.0)) {
        v->status = ORC_ETRAPPED;
        return false;
    }
    double u1, u2;
    event_uniforms(v->seed, v->uid, v->n, &u1, &u2);
    double t = u1 * R;
    int slot, dir;
    select_event(v, t, &slot, &dir);
    if (v->debug & 2) {
        double margin;
        int e_tree = 8 * slot + dir;
        int e_scan = scan_select(v, t, &margin);
        if (e_scan != e_tree) {
            if (margin / R < 1e-12) v->cnt[1]++; else v->cnt[2]++;
        }
    }
    // (a7) swap: sigma_w <- A, sigma_m <- V; vacancy slot moves to m.
    int w = v->pos[slot];
    int dx, dy, dz;
    dirvec(dir, dx, dy, dz);
    int m = nbr(v, w, dx, dy, dz);
    int A = v->sp[m];
    v->sp[w] = (uint8_t)A;
    v->sp[m] = (uint8_t)VAC;
    v->pos[slot] = m;
    v->disp[3 * slot + 0] += dx;
    v->disp[3 * slot + 1] += dy;
    v->disp[3 * slot + 2] += dz;
    if (v->model == 1) {
        const Shells& S = shells();
        for (const Off& o : S.sph) v->rho[nbr(v, w, o.dx, o.dy, o.dz)] += v->fq[A][o.shell];
        for (const Off& o : S.sph) v->rho[nbr(v, m, o.dx, o.dy, o.dz)] -= v->fq[A][o.shell];
    }
    if (v->debug & 8) {
        for (int c = 0; c < 3; ++c) {
            int d = c == 0 ? dx : (c == 1 ? dy : dz);
            v->tdisp[3 * w + c] = v->tdisp[3 * m + c] - d;
            v->tdisp[3 * m + c] = 0;
        }
    }
    // (a9) clock: dt = -ln(u2)/R, Neumaier-compensated (t_hi, t_lo).
    double dt = -std::log(u2) / R;
    double s = v->t_hi + dt;
    if (std::fabs(v->t_hi) >= std::fabs(dt))
        v->t_lo += (v->t_hi - s) + dt;
    else
        v->t_lo += (dt - s) + v->t_hi;
    v->t_hi = s;
    if (log_entry) *log_entry = 8 * slot + dir;
    if (dt_entry) *dt_entry = dt;
    v->n++;
    // (a8) refresh the moved vacancy and every vacancy whose read set changed.
    v->numeric = 0;
    for (int q = 0; q < v->nv; ++q)
        if (q == slot || affected(v, v->pos[q], w, m)) refresh_vacancy(v, q);
    if (v->numeric) v->status = ORC_ENUMERIC;
    if (v->debug) debug_checks(v);
    return true;
}

// ---- synchronous sublattice schedule (intra-voxel parallel AKMC) -----------------
// The voxel is cut into sectors of S^3 cells, each into 8 octants of (S/2)^3.
// Superstep k evolves octant k mod 8 (bit 0: x half, bit 1: y, bit 2: z) of
// every sector; each active octant runs its own KMC over the vacancies that
// lie in it at the start of the superstep, with its own clock starting at 0,
// until the next event's time would pass the window T (that event is not
// made); a vacancy that leaves the octant takes no further part in the
// superstep.  The reads of an event reach 4 half units beyond its vacancy and
// its writes 4 half units beyond the vacancy's start (hop 1 + cutoff sphere
// 3), while active octants of one superstep are S + 1 half units apart, so
// for S >= 8 no event of one octant reads or writes what another octant's
// events touch and their order does not matter; this serial schedule takes
// them in sector order.  One cycle of 8 supersteps evolves every region for
// T (a first-order splitting of the voxel's master equation into octant
// parts), so the voxel's clock advances by T/8 per superstep.
void sl_uniforms(uint64_t seed, uint64_t uid, uint32_t i, uint32_t k, uint32_t sector, double* u1, double* u2) {
    uint32_t ctr[4] = {i, k, sector, 0xC0000000u | ((uint32_t)uid & 0x3FFFFFFFu)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    philox(ctr, key, x);
    uint64_t a = ((uint64_t)x[0] << 21) | (x[1] >> 11);
    uint64_t b = ((uint64_t)x[2] << 21) | (x[3] >> 11);
    *u1 = (double)a * 0x1p-53;
    *u2 = (double)(b + 1) * 0x1p-53;
}

bool in_octant(const orc_voxel* v, int site, int S, int sx, int sy, int sz, int oct) {
    int X, Y, Z;
    coords_of(v, site, X, Y, Z);
    const int x = X >> 1, y = Y >> 1, z = Z >> 1, h = S / 2;
    const int lx = x - sx * S - (oct & 1) * h, ly = y - sy * S - ((oct >> 1) & 1) * h,
              lz = z - sz * S - ((oct >> 2) & 1) * h;
    return lx >= 0 && lx < h && ly >= 0 && ly < h && lz >= 0 && lz < h;
}

// The hop (slot, dir): swap, densities, displacement, tracers, refresh of every
// affected vacancy (as in one_event).
void apply_hop(orc_voxel* v, int slot, int dir) {
    int w = v->pos[slot];
    int dx, dy, dz;
    dirvec(dir, dx, dy, dz);
    int m = nbr(v, w, dx, dy, dz);
    int A = v->sp[m];
    v->sp[w] = (uint8_t)A;
    v->sp[m] = (uint8_t)VAC;
    v->pos[slot] = m;
    v->disp[3 * slot + 0] += dx;
    v->disp[3 * slot + 1] += dy;
    v->disp[3 * slot + 2] += dz;
    if (v->model == 1) {
        const Shells& S = shells();
        for (const Off& o : S.sph) v->rho[nbr(v, w, o.dx, o.dy, o.dz)] += v->fq[A][o.shell];
        for (const Off& o : S.sph) v->rho[nbr(v, m, o.dx, o.dy, o.dz)] -= v->fq[A][o.shell];
    }
    if (v->debug & 8) {
        for (int c = 0; c < 3; ++c) {
            int d = c == 0 ? dx : (c == 1 ? dy : dz);
            v->tdisp[3 * w + c] = v->tdisp[3 * m + c] - d;
            v->tdisp[3 * m + c] = 0;
        }
    }
    v->n++;
    v->numeric = 0;
    for (int q = 0; q < v->nv; ++q)
        if (q == slot || affected(v, v->pos[q], w, m)) refresh_vacancy(v, q);
    if (v->numeric) v->status = ORC_ENUMERIC;
}

uint64_t sl_octant(orc_voxel* v, uint32_t k, int S, int sid, int oct) {
    const int ns = v->L / S;
    const int sx = sid % ns, sy = (sid / ns) % ns, sz = sid / (ns * ns);
    std::vector<int> act;
    for (int q = 0; q < v->nv; ++q)
        if (in_octant(v, v->pos[q], S, sx, sy, sz, oct)) act.push_back(q);
    if (act.empty()) return 0;
    std::vector<char> on(act.size(), 1);
    int P = 1;
    while (P < (int)act.size()) P <<= 1;
    std::vector<double> tree(2 * P, 0.0);
    double t = 0.0;
    uint32_t i = 0;
    uint64_t made = 0;
    for (;;) {
        if (v->status != ORC_OK) break;
        std::fill(tree.begin(), tree.end(), 0.0);
        for (size_t j = 0; j < act.size(); ++j)
            tree[P + j] = on[j] ? vacancy_sum(&v->rate[8 * act[j]]) : 0.0;
        for (int n = P - 1; n >= 1; --n) tree[n] = tree[2 * n] + tree[2 * n + 1];
        const double R = tree[1];
        if (!(R > 0.0)) break;
        double u1, u2;
        sl_uniforms(v->seed, v->uid, i, k, (uint32_t)sid, &u1, &u2);
        const double dt = -std::log(u2) / R;
        if (t + dt > v->sl_T) break;
        double tt = u1 * R;
        const int j = descend(tree.data(), P, tt);
        const double* g = &v->rate[8 * act[j]];
        double h[16];
        for (int d = 0; d < 8; ++d) h[8 + d] = g[d];
        for (int n = 7; n >= 1; --n) h[n] = h[2 * n] + h[2 * n + 1];
        const int dir = descend(h, 8, tt);
        apply_hop(v, act[j], dir);
        if (!in_octant(v, v->pos[act[j]], S, sx, sy, sz, oct)) on[j] = 0;
        t += dt;
        ++i;
        ++made;
    }
    return made;
}

int init_model(orc_voxel* v, const orc_model* m) {
    std::memcpy(v->eps1, m->eps1, sizeof v->eps1);
    std::memcpy(v->eps2, m->eps2, sizeof v->eps2);
    std::memcpy(v->E0, m->E0, sizeof v->E0);
    v->nu = m->nu;
    v->a = m->a;
    if (v->model == 1) {
        if (m->n_r < 2 || m->n_rho < 2 || !m->phi_tab || !m->f_tab || !m->F_tab) return ORC_EINVAL;
        v->shift = rho_shift(m->rho_h);
        if (v->shift < 0) return ORC_EINVAL;
        v->n_rho = m->n_rho;
        v->rho_h = m->rho_h;
        v->F_tab.assign(m->F_tab, m->F_tab + (size_t)4 * m->n_rho * 2);
        double ph[50];
        int64_t fq[20];
        int st = orc_shell_constants(m, ph, fq);
        if (st) return st;
        for (int p = 0; p < 10; ++p) {
            v->phi_s[p][0] = 0.0;
            for (int s = 1; s <= 5; ++s) v->phi_s[p][s] = ph[p * 5 + s - 1];
        }
        for (int b = 0; b < 4; ++b) {
            v->fq[b][0] = 0;
            for (int s = 1; s <= 5; ++s) v->fq[b][s] = fq[b * 5 + s - 1];
        }
    }
    return ORC_OK;
}

}  // namespace

extern "C" {

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    philox(ctr, key, out);
}

void orc_event_uniforms(uint64_t seed, uint64_t uid, uint64_t n, double* u1, double* u2) {
    event_uniforms(seed, uid, n, u1, u2);
}

int orc_shell_constants(const orc_model* m, double phi_out[50], int64_t fq_out[20]) {
    if (m->n_r < 2 || !m->phi_tab || !m->f_tab) return ORC_EINVAL;
    for (int s = 1; s <= 5; ++s) {
        double r = (m->a * 0.5) * std::sqrt((double)SHELL_LEN2[s]);
        if (!(r < m->r_cut)) return ORC_EINVAL;
        for (int p = 0; p < 10; ++p)
            phi_out[p * 5 + s - 1] = table_at_r(m->phi_tab + (size_t)p * m->n_r * 2, m->n_r, m->r_cut, r);
        for (int b = 0; b < 4; ++b) {
            double f = table_at_r(m->f_tab + (size_t)b * m->n_r * 2, m->n_r, m->r_cut, r);
            fq_out[b * 5 + s - 1] = std::llround(f * (double)(1 << RHO_BITS));
        }
    }
    return ORC_OK;
}

double orc_embed(const orc_model* m, int a, int64_t rho_fixed, int* err) {
    orc_voxel tmp;
    tmp.shift = rho_shift(m->rho_h);
    tmp.n_rho = m->n_rho;
    tmp.rho_h = m->rho_h;
    tmp.F_tab.assign(m->F_tab, m->F_tab + (size_t)4 * m->n_rho * 2);
    double e = embed(&tmp, a, rho_fixed);
    if (err) *err = tmp.numeric;
    return e;
}

orc_voxel* orc_create(const orc_desc* d, const orc_model* m, int* status) {
    int st = ORC_OK;
    if (d->model == 0 && d->L < 3) st = ORC_EINVAL;
    if (d->model == 1 && d->L < 4) st = ORC_EINVAL;
    if (d->model != 0 && d->model != 1) st = ORC_EINVAL;
    if (d->n_vac < 1 || !(d->T > 0.0) || d->L > 1024) st = ORC_EINVAL;
    if (st) { if (status) *status = st; return nullptr; }
    orc_voxel* v = new orc_voxel();
    v->L = d->L;
    v->N = 2 * d->L * d->L * d->L;
    v->nv = d->n_vac;
    v->model = d->model;
    v->T = d->T;
    v->beta = 1.0 / (KB * d->T);
    v->seed = d->seed;
    v->uid = d->uid;
    st = init_model(v, m);
    // (a1) species counts n_s = floor(frac_s * N + 0.5), Fe the balance.
    int64_t cnt[3];
    int64_t total = d->n_vac;
    for (int s = 0; s < 3; ++s) {
        cnt[s] = (int64_t)std::floor(d->frac[s] * (double)v->N + 0.5);
        if (cnt[s] < 0) st = ORC_EINVAL;
        total += cnt[s];
    }
    if (total > v->N) st = ORC_EINVAL;
    if (st) { delete v; if (status) *status = st; return nullptr; }
    v->sp.assign(v->N, (uint8_t)FE);
    v->stamp.assign(v->N, 0u);
    // Placement by sequential rejection: draw k gives a uniform site; it is
    // taken if it still holds Fe.  Order: vacancies (slot = placement order), Cu, Ni, Mn.
    uint64_t k = 0;
    auto place = [&](int species, int64_t count) {
        for (int64_t c = 0; c < count; ++c) {
            for (;;) {
                int s = placement_draw(v->seed, v->uid, k++, v->N);
                if (v->sp[s] == FE) {
                    v->sp[s] = (uint8_t)species;
                    if (species == VAC) v->pos.push_back(s);
                    break;
                }
            }
        }
    };
    place(VAC, d->n_vac);
    place(1, cnt[0]);
    place(2, cnt[1]);
    place(3, cnt[2]);
    v->disp.assign(3 * (size_t)v->nv, 0);
    v->tdisp.assign(3 * (size_t)v->N, 0);
    rebuild_all(v);
    if (status) *status = v->status;
    return v;
}

void orc_destroy(orc_voxel* v) { delete v; }

int orc_load(orc_voxel* v, const uint8_t* species, const int32_t* vac_pos, int32_t n_vac,
             double t_hi, double t_lo, uint64_t n_events) {
    if (n_vac < 1) return ORC_EINVAL;
    int nvac_lattice = 0;
    for (int i = 0; i < v->N; ++i) {
        if (species[i] > VAC) return ORC_EINVAL;
        nvac_lattice += species[i] == VAC;
    }
    if (nvac_lattice != n_vac) return ORC_EINVAL;
    for (int q = 0; q < n_vac; ++q)
        if (vac_pos[q] < 0 || vac_pos[q] >= v->N || species[vac_pos[q]] != VAC) return ORC_EINVAL;
    v->sp.assign(species, species + v->N);
    v->nv = n_vac;
    v->pos.assign(vac_pos, vac_pos + n_vac);
    v->disp.assign(3 * (size_t)n_vac, 0);
    v->tdisp.assign(3 * (size_t)v->N, 0);
    v->t_hi = t_hi;
    v->t_lo = t_lo;
    v->n = n_events;
    v->status = ORC_OK;
    rebuild_all(v);
    return v->status;
}

int orc_step(orc_voxel* v, uint64_t n, int32_t* log, double* dt_log) {
    for (uint64_t i = 0; i < n; ++i) {
        if (v->status != ORC_OK) break;
        if (!one_event(v, log ? log + i : nullptr, dt_log ? dt_log + i : nullptr)) break;
    }
    return v->status;
}

int orc_step_sublattice(orc_voxel* v, uint64_t k0, uint32_t n_supersteps, int32_t S, double T, int32_t reverse,
                        uint64_t* events) {
    if (S < 8 || S % 2 || v->L % S || !(T > 0.0)) return ORC_EINVAL;
    const int ns = v->L / S, n_sec = ns * ns * ns;
    v->sl_T = T;
    for (uint32_t st = 0; st < n_supersteps; ++st) {
        if (v->status != ORC_OK) break;
        const uint32_t k = (uint32_t)(k0 + st);
        const int oct = (int)(k % 8);
        uint64_t made = 0;
        for (int idx = 0; idx < n_sec; ++idx) {
            const int sid = reverse ? n_sec - 1 - idx : idx;
            made += sl_octant(v, k, S, sid, oct);
        }
        const double dt = T * 0.125;
        double s2 = v->t_hi + dt;
        if (std::fabs(v->t_hi) >= std::fabs(dt))
            v->t_lo += (v->t_hi - s2) + dt;
        else
            v->t_lo += (dt - s2) + v->t_hi;
        v->t_hi = s2;
        if (events) events[st] = made;
    }
    return v->status;
}

int orc_get(const orc_voxel* v, uint8_t* species, int32_t* vac_pos, int32_t* vac_disp,
            double* rates, double* dE, double* t_hi, double* t_lo, uint64_t* n_events) {
    if (species) std::memcpy(species, v->sp.data(), v->N);
    if (vac_pos) for (int q = 0; q < v->nv; ++q) vac_pos[q] = v->pos[q];
    if (vac_disp) for (int q = 0; q < 3 * v->nv; ++q) vac_disp[q] = v->disp[q];
    if (rates) for (int q = 0; q < 8 * v->nv; ++q) rates[q] = v->rate[q];
    if (dE) for (int q = 0; q < 8 * v->nv; ++q) dE[q] = v->dE[q];
    if (t_hi) *t_hi = v->t_hi;
    if (t_lo) *t_lo = v->t_lo;
    if (n_events) *n_events = v->n;
    return v->status;
}

int32_t orc_n_sites(const orc_voxel* v) { return v->N; }
int32_t orc_n_vac(const orc_voxel* v) { return v->nv; }
double orc_total_rate(const orc_voxel* v) { return v->tree[1]; }

double orc_energy(const orc_voxel* v) {
    return v->model == 0 ? energy_pair(v, v->sp.data()) : energy_eam(v, v->sp.data());
}

double orc_hop_de_local(const orc_voxel* v, int slot, int dir) {
    int w = v->pos[slot], m = hop_target(v, w, dir);
    if (v->sp[m] == VAC) return 0.0;
    return v->model == 0 ? de_pair_local(v, v->sp.data(), w, m)
                         : de_eam_local(v, v->sp.data(), v->rho.data(), w, m);
}

// Brute force: per-site energy after minus before, summed over the whole lattice.
double orc_hop_de_brute(const orc_voxel* v, int slot, int dir) {
    int w = v->pos[slot], m = hop_target(v, w, dir);
    if (v->sp[m] == VAC) return 0.0;
    std::vector<uint8_t> after(v->sp);
    after[w] = after[m];
    after[m] = (uint8_t)VAC;
    if (v->model == 0) return energy_pair(v, after.data()) - energy_pair(v, v->sp.data());
    double de = 0.0;
    for (int i = 0; i < v->N; ++i)
        de += site_energy_eam(v, after.data(), i) - site_energy_eam(v, v->sp.data(), i);
    return de;
}

double orc_hop_rate(const orc_voxel* v, int slot, int dir) {
    double de;
    return hop_rate_de(v, slot, dir, &de);
}

int64_t orc_rho_fixed(const orc_voxel* v, int site) { return rho_scratch(v, v->sp.data(), site); }

void orc_rho_all(const orc_voxel* v, int64_t* out) {
    for (int i = 0; i < v->N; ++i) out[i] = rho_scratch(v, v->sp.data(), i);
}

void orc_set_debug(orc_voxel* v, int flags) { v->debug = flags; }

void orc_debug_counts(const orc_voxel* v, uint64_t out[5]) {
    for (int i = 0; i < 5; ++i) out[i] = v->cnt[i];
}

double orc_tracer_r2(const orc_voxel* v) {
    double s = 0.0;
    for (int i = 0; i < v->N; ++i) {
        if (v->sp[i] == VAC) continue;
        const int* d = &v->tdisp[3 * (size_t)i];
        s += (double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2];
    }
    return s;
}

// Connected components of Cu (species 1) by breadth-first search.
int32_t orc_cluster_hist(const orc_voxel* v, int mode, int64_t hist[8], int32_t* sizes_out) {
    const Shells& S = shells();
    std::vector<Off> adj;
    for (const Off& o : S.n12)
        if (mode == 0 || o.shell == 1) adj.push_back(o);
    for (int b = 0; b < 8; ++b) hist[b] = 0;
    std::vector<char> seen(v->N, 0);
    std::vector<int> queue;
    int32_t nc = 0;
    for (int i = 0; i < v->N; ++i) {
        if (v->sp[i] != 1 || seen[i]) continue;
        queue.clear();
        queue.push_back(i);
        seen[i] = 1;
        for (size_t q = 0; q < queue.size(); ++q)
            for (const Off& o : adj) {
                int j = nbr(v, queue[q], o.dx, o.dy, o.dz);
                if (v->sp[j] == 1 && !seen[j]) { seen[j] = 1; queue.push_back(j); }
            }
        int sz = (int)queue.size();
        int bin = sz <= 4 ? sz - 1 : (sz < 10 ? 4 : (sz < 20 ? 5 : (sz < 50 ? 6 : 7)));
        hist[bin]++;
        if (sizes_out) sizes_out[nc] = sz;
        nc++;
    }
    return nc;
}

}  // extern "C"
