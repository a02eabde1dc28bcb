// k_select.cu -- global masked softmax sampling over segments of logits
// (the action distribution of Eq. 1-2: logits z of every candidate transition
// of every agent, scaled by 1/tau where admissible and -inf elsewhere, one
// global softmax per segment, one transition drawn from it).
//
// A segment is one system (one voxel): the concatenated logits of all of its
// agents.  It is cut into parts of at most 8192 logits (4 tiles of 2048).
//   1. One CTA per part reads the part once (16-byte loads where aligned) into
//      registers, takes its maximum m_p of z/tau (z * (1/tau), rounded once)
//      and its weights q = rn(exp(z/tau - m_p) 2^32) (FP32 exp), summed exactly
//      in int64 per tile and per part (S_p).
//   2. One CTA per segment: M = max m_p; part weights w_p = rn(S_p exp(m_p - M))
//      (integers); t = floor(u W) for W = sum w_p and the segment's uniform u;
//      the part whose running sum of w first exceeds t; inside it t scaled to
//      the part's own units, floor((t - before) S_p / w_p); then the tile and
//      the logit whose running sum of q first exceeds that.  Every sum is an
//      exact integer, so the draw does not depend on the launch shape, and a
//      segment of one part is an exact inverse-CDF draw over its q.
#include <akmc.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "akmc_device.cuh"
#include "akmc_launch.h"

namespace akmc {
namespace {

constexpr int kSelThreads = 256;
constexpr int kSelPerThread = 8;
constexpr int kSelTile = kSelThreads * kSelPerThread;   // 2048 logits
constexpr int kSelTilesPerPart = 4;
constexpr int64_t kSelPart = (int64_t)kSelTile * kSelTilesPerPart;   // 8192 logits
constexpr int kSelGroups = kSelPart / (4 * kSelThreads);              // float4 groups per thread (8)
constexpr int64_t kSelMaxSegment = (int64_t)1 << 30;
constexpr float kFix = 4294967296.0f;                   // weights in units of 2^-32
constexpr uint32_t kSelStream = 0x53454c45u;            // Philox counter word 3 of the draws

struct SelPart {
    int64_t begin, end;   // logits [begin, end) of the flat array
    int32_t seg, first;   // segment, index of the segment's first part
};

struct SelSeg {
    int64_t begin;        // first logit of the segment
    int32_t first_part, n_parts;
};

struct SelHeader {
    int32_t n_seg, n_parts;
};

struct SelLayout {
    size_t header, segs, parts, pmax, psum, tsum, total;
};

SelLayout sel_layout(int n_seg, int n_parts) {
    SelLayout l;
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o = (o + b + 255) / 256 * 256; return at; };
    l.header = take(sizeof(SelHeader));
    l.segs = take(sizeof(SelSeg) * (size_t)n_seg);
    l.parts = take(sizeof(SelPart) * (size_t)n_parts);
    l.pmax = take(sizeof(float) * (size_t)n_parts);
    l.psum = take(sizeof(long long) * (size_t)n_parts);
    l.tsum = take(sizeof(long long) * (size_t)n_parts * kSelTilesPerPart);
    l.total = o;
    return l;
}

// Admissible iff the mask (when given) is nonzero and the logit is finite (a
// logit of -inf is the masked value of Eq. 1).  The scaled logit is z * (1/tau)
// (rounded once; every pass uses the same expression).
__device__ __forceinline__ bool sel_ok(float v, uint32_t mbyte) { return mbyte != 0 && isfinite(v); }

__device__ __forceinline__ float block_max(float v, float* sm) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < kSelThreads / 32 ? sm[threadIdx.x] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) sm[0] = v;
    }
    __syncthreads();
    v = sm[0];
    __syncthreads();
    return v;
}

__device__ __forceinline__ long long block_sum(long long v, long long* sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < kSelThreads / 32 ? sm[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sm[0] = v;
    }
    __syncthreads();
    v = sm[0];
    __syncthreads();
    return v;
}

__device__ __forceinline__ long long sel_weight(float v, bool ok, float inv_tau, float M) {
    return ok ? __float2ll_rn(expf(v * inv_tau - M) * kFix) : 0;
}

// One CTA per part: the part's logits in registers (thread i holds the 4
// consecutive logits at begin + 1024 g + 4 i of every group g), the part
// maximum m_p of the scaled logits (the maximum of the raw admissible logits
// times 1/tau: multiplication by a positive constant keeps the order), and the
// exact tile and part sums of q = rn(exp(z/tau - m_p) 2^32).  Tile k holds
// groups 2k and 2k + 1.
__global__ void __launch_bounds__(kSelThreads, 4) sel_part_kernel(const float* z, const uint8_t* mask, float inv_tau,
                                                               const SelPart* parts, float* pmax, long long* psum,
                                                               long long* tsum) {
    __shared__ float smf[32];
    __shared__ long long sml[kSelThreads / 32][kSelTilesPerPart];
    const SelPart P = parts[blockIdx.x];
    const int tid = threadIdx.x;
    const bool vec = (((uintptr_t)(z + P.begin)) & 15) == 0 &&
                     (mask == nullptr || (((uintptr_t)(mask + P.begin)) & 3) == 0);
    float v[4 * kSelGroups];
    uint32_t mb[kSelGroups];
#pragma unroll
    for (int g = 0; g < kSelGroups; ++g) {
        const int64_t jj = P.begin + (int64_t)g * (4 * kSelThreads) + 4 * tid;
        if (vec && jj + 3 < P.end) {
            const float4 f = *(const float4*)(z + jj);
            v[4 * g] = f.x;
            v[4 * g + 1] = f.y;
            v[4 * g + 2] = f.z;
            v[4 * g + 3] = f.w;
            mb[g] = mask ? *(const uint32_t*)(mask + jj) : 0x01010101u;
        } else {
            uint32_t m = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t j = jj + i;
                v[4 * g + i] = j < P.end ? z[j] : -INFINITY;
                m |= (j < P.end ? (mask ? (uint32_t)mask[j] : 1u) : 0u) << (8 * i);
            }
            mb[g] = m;
        }
    }
    float m = -INFINITY;
#pragma unroll
    for (int g = 0; g < kSelGroups; ++g)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (sel_ok(v[4 * g + i], (mb[g] >> (8 * i)) & 0xFFu)) m = fmaxf(m, v[4 * g + i]);
    const float mp = block_max(m, smf) * inv_tau;
    // the four tile sums, reduced together (warp shuffles, then one pass over the warps)
    long long sk[kSelTilesPerPart];
#pragma unroll
    for (int k = 0; k < kSelTilesPerPart; ++k) {
        sk[k] = 0;
        if (mp > -INFINITY) {
#pragma unroll
            for (int g = 2 * k; g < 2 * k + 2; ++g)
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    sk[k] += sel_weight(v[4 * g + i], sel_ok(v[4 * g + i], (mb[g] >> (8 * i)) & 0xFFu), inv_tau, mp);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sk[k] += __shfl_xor_sync(0xffffffffu, sk[k], o);
    }
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kSelTilesPerPart; ++k) sml[warp][k] = sk[k];
    __syncthreads();
    if (tid < kSelTilesPerPart) {
        long long t = 0;
        for (int w = 0; w < kSelThreads / 32; ++w) t += sml[w][tid];
        tsum[(size_t)blockIdx.x * kSelTilesPerPart + tid] = t;
        const long long p1 = t + __shfl_xor_sync(0xfu, t, 1);
        const long long p2 = p1 + __shfl_xor_sync(0xfu, p1, 2);
        if (tid == 0) {
            pmax[blockIdx.x] = mp;
            psum[blockIdx.x] = p2;
        }
    }
}

// Exclusive prefix over the CTA of one int64 per thread (fixed order), and the total.
__device__ __forceinline__ long long block_excl_scan(long long v, long long* sm, long long& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sm[warp] = incl;
    __syncthreads();
    long long before = 0, tot = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) {
        if (w < warp) before += sm[w];
        tot += sm[w];
    }
    __syncthreads();
    total = tot;
    return before + incl - v;
}

// Integer weight of part p of a segment with maximum M: rn(S_p exp(m_p - M))
// (exactly S_p when m_p = M).
__device__ __forceinline__ long long part_weight(long long Sp, float mp, float M) {
    if (Sp == 0 || !(mp > -INFINITY)) return 0;
    return llrint((double)Sp * exp((double)mp - (double)M));
}

// One CTA per segment.
__global__ void __launch_bounds__(kSelThreads) sel_pick_kernel(const float* z, const uint8_t* mask, float inv_tau,
                                                               const SelSeg* segs, const SelPart* parts,
                                                               const float* pmax, const long long* psum,
                                                               const long long* tsum, uint64_t seed, uint64_t ctr,
                                                               int64_t* out_index, float* out_logp) {
    __shared__ float smf[32];
    __shared__ long long sml[32];
    __shared__ int64_t s_tile;
    __shared__ long long s_rest, s_t;
    __shared__ int s_part;
    const int s_id = blockIdx.x;
    const SelSeg S = segs[s_id];
    const int tid = threadIdx.x;
    const int np = S.n_parts;
    // segment maximum and the parts' integer weights (thread tid owns the
    // consecutive parts [c0, c1))
    float m = -INFINITY;
    for (int p = tid; p < np; p += kSelThreads) m = fmaxf(m, pmax[S.first_part + p]);
    const float M = block_max(m, smf);
    const int C = (np + kSelThreads - 1) / kSelThreads;
    const int c0 = min(np, tid * C), c1 = min(np, c0 + C);
    long long own = 0;
    for (int p = c0; p < c1; ++p) own += part_weight(psum[S.first_part + p], pmax[S.first_part + p], M);
    long long W = 0;
    const long long excl = block_excl_scan(own, sml, W);
    if (W <= 0) {
        if (tid == 0) {
            out_index[s_id] = -1;
            out_logp[s_id] = NAN;
        }
        return;
    }
    if (tid == 0) {
        // u = m 2^-53 from the segment's Philox block, t = floor(u W) exactly
        uint32_t x0 = (uint32_t)ctr, x1 = (uint32_t)(ctr >> 32), x2 = (uint32_t)s_id, x3 = kSelStream;
        philox4x32_10(x0, x1, x2, x3, (uint32_t)seed, (uint32_t)(seed >> 32));
        const unsigned long long u53 = ((unsigned long long)x0 << 21) | (x1 >> 11);
        const unsigned __int128 prod = (unsigned __int128)u53 * (unsigned long long)W;
        s_t = (long long)(prod >> 53);
    }
    __syncthreads();
    const long long t = s_t;
    if (t >= excl && t < excl + own) {
        // this thread's parts hold t: the part, then t in the part's own units
        long long r = t - excl;
        int p = c0;
        for (; p < c1 - 1; ++p) {
            const long long w = part_weight(psum[S.first_part + p], pmax[S.first_part + p], M);
            if (r < w) break;
            r -= w;
        }
        const int gp = S.first_part + p;
        const long long Sp = psum[gp];
        const long long w = part_weight(Sp, pmax[gp], M);
        long long ti = (long long)(((unsigned __int128)r * (unsigned long long)Sp) / (unsigned long long)w);
        ti = min(ti, Sp - 1);
        int k = 0;
        while (k < kSelTilesPerPart - 1 && ti >= tsum[(size_t)gp * kSelTilesPerPart + k])
            ti -= tsum[(size_t)gp * kSelTilesPerPart + k++];
        s_part = gp;
        s_tile = parts[gp].begin + (int64_t)k * kSelTile;
        s_rest = ti;
    }
    __syncthreads();
    const int gp = s_part;
    const float mp = pmax[gp];
    const int64_t part_end = parts[gp].end;
    // the tile's logits in order: thread i takes 8 consecutive ones
    const int64_t j0 = s_tile + (int64_t)tid * kSelPerThread;
    long long q[kSelPerThread];
    float zq[kSelPerThread];
    long long mine = 0;
#pragma unroll
    for (int i = 0; i < kSelPerThread; ++i) {
        const int64_t j = j0 + i;
        q[i] = 0;
        zq[i] = 0.f;
        if (j < part_end) {
            const float v = z[j];
            const bool ok = sel_ok(v, mask ? (uint32_t)mask[j] : 1u);
            zq[i] = v * inv_tau;
            q[i] = sel_weight(v, ok, inv_tau, mp);
        }
        mine += q[i];
    }
    long long tile_total = 0;
    const long long before = block_excl_scan(mine, sml, tile_total);
    const long long r = s_rest;
    if (r >= before && r < before + mine) {
        long long rr = r - before;
        int i = 0;
        while (i < kSelPerThread - 1 && rr >= q[i]) rr -= q[i++];
        out_index[s_id] = j0 + i - S.begin;
        out_logp[s_id] = (float)((double)(zq[i] - M) - log((double)W * 0x1p-32));
    }
}

akmc_status sel_fail(akmc_status st, const std::string& msg) {
    set_last_error(msg.c_str());
    return st;
}

bool sel_plan(const int64_t* off, int n_seg, std::vector<SelSeg>& segs, std::vector<SelPart>& parts,
              std::string& err) {
    segs.clear();
    parts.clear();
    for (int s = 0; s < n_seg; ++s) {
        const int64_t b = off[s], e = off[s + 1];
        if (e < b) {
            err = "segment " + std::to_string(s) + " has a negative length";
            return false;
        }
        if (e - b > kSelMaxSegment) {
            err = "segment " + std::to_string(s) + " longer than 2^30 logits";
            return false;
        }
        SelSeg S;
        S.begin = b;
        S.first_part = (int32_t)parts.size();
        const int64_t n = e - b;
        const int np = n == 0 ? 1 : (int)((n + kSelPart - 1) / kSelPart);
        S.n_parts = np;
        for (int p = 0; p < np; ++p) {
            SelPart P;
            P.begin = b + (int64_t)p * kSelPart;
            P.end = std::min(e, P.begin + kSelPart);
            if (P.begin > e) P.begin = e;
            P.seg = s;
            P.first = S.first_part;
            parts.push_back(P);
        }
        segs.push_back(S);
    }
    return true;
}

}  // namespace
}  // namespace akmc

extern "C" size_t akmc_select_scratch_bytes(const int64_t* host_offsets, int32_t n_seg) {
    using namespace akmc;
    if (!host_offsets || n_seg < 1) return 0;
    std::vector<SelSeg> segs;
    std::vector<SelPart> parts;
    std::string err;
    if (!sel_plan(host_offsets, n_seg, segs, parts, err)) return 0;
    return sel_layout(n_seg, (int)parts.size()).total;
}

extern "C" akmc_status akmc_select_plan(const int64_t* host_offsets, int32_t n_seg, void* scratch, size_t bytes,
                                        int32_t* n_parts_out, akmc_stream stream) {
    using namespace akmc;
    if (!host_offsets || !scratch || !n_parts_out) return sel_fail(AKMC_EINVAL, "NULL argument");
    if (n_seg < 1) return sel_fail(AKMC_EINVAL, "need at least one segment");
    if ((uintptr_t)scratch % 256) return sel_fail(AKMC_EINVAL, "scratch must be 256-byte aligned");
    std::vector<SelSeg> segs;
    std::vector<SelPart> parts;
    std::string err;
    if (!sel_plan(host_offsets, n_seg, segs, parts, err)) return sel_fail(AKMC_EINVAL, err);
    const SelLayout l = sel_layout(n_seg, (int)parts.size());
    if (bytes < l.total)
        return sel_fail(AKMC_ENOMEM, "scratch has " + std::to_string(bytes) + " bytes, plan needs " +
                                         std::to_string(l.total));
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)scratch;
    SelHeader h{n_seg, (int32_t)parts.size()};
    cudaError_t e = cudaMemcpyAsync(base + l.header, &h, sizeof h, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + l.segs, segs.data(), sizeof(SelSeg) * segs.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + l.parts, parts.data(), sizeof(SelPart) * parts.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host vectors must outlive the copies
    if (e != cudaSuccess) return sel_fail(AKMC_ECUDA, std::string("plan upload: ") + cudaGetErrorString(e));
    *n_parts_out = (int32_t)parts.size();
    return AKMC_OK;
}

extern "C" akmc_status akmc_select_logits(const float* logits, const uint8_t* mask, int32_t n_seg, int32_t n_parts,
                                          float tau, uint64_t seed, uint64_t counter, const void* scratch,
                                          int64_t* out_index, float* out_logp, akmc_stream stream) {
    using namespace akmc;
    if (!logits || !scratch || !out_index || !out_logp) return sel_fail(AKMC_EINVAL, "NULL argument");
    if (n_seg < 1 || n_parts < n_seg) return sel_fail(AKMC_EINVAL, "n_seg / n_parts do not match a plan");
    if (!(tau > 0.f) || !std::isfinite(tau)) return sel_fail(AKMC_EINVAL, "tau must be positive and finite");
    const SelLayout l = sel_layout(n_seg, n_parts);
    char* base = (char*)scratch;
    const SelSeg* segs = (const SelSeg*)(base + l.segs);
    const SelPart* parts = (const SelPart*)(base + l.parts);
    float* pmax = (float*)(base + l.pmax);
    long long* psum = (long long*)(base + l.psum);
    long long* tsum = (long long*)(base + l.tsum);
    cudaStream_t st = (cudaStream_t)stream;
    const float inv_tau = 1.0f / tau;
    sel_part_kernel<<<n_parts, kSelThreads, 0, st>>>(logits, mask, inv_tau, parts, pmax, psum, tsum);
    sel_pick_kernel<<<n_seg, kSelThreads, 0, st>>>(logits, mask, inv_tau, segs, parts, pmax, psum, tsum, seed,
                                                   counter, out_index, out_logp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sel_fail(AKMC_ECUDA, std::string("select kernels: ") + cudaGetErrorString(e));
    return AKMC_OK;
}
