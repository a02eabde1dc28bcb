// k_select.cu -- global masked softmax sampling over segments of logits
// (the action distribution of Eq. 1-2: logits z of every candidate transition
// of every agent, scaled by 1/tau where admissible and -inf elsewhere, one
// global softmax per segment, one transition drawn from it).
//
// A segment is one system (one voxel): the concatenated logits of all of its
// agents.  Three stream-ordered launches, each spread over "parts" of at most
// 65536 logits so that long and short segments balance across the SMs:
//   1. part maxima of z/tau over admissible entries;
//   2. with the segment maximum M, the weights w = exp(z/tau - M) (FP32 exp)
//      in fixed point q = rn(w 2^32), summed exactly per 2048-logit tile and
//      per part (int64; the sums do not depend on the summation order, so the
//      draw does not depend on the launch shape);
//   3. per segment: W = sum of q, t = floor(u W) for the segment's uniform u,
//      then the part, the tile and the logit whose running sum first exceeds t
//      (inverse-CDF search over the exact integer prefix sums).
// Logits are read coalesced (one warp reads 32 consecutive logits per load).
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
constexpr int kSelTilesPerPart = 32;
constexpr int64_t kSelPart = (int64_t)kSelTile * kSelTilesPerPart;   // 65536 logits
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
// logit of -inf is the masked value of Eq. 1).
__device__ __forceinline__ bool sel_load(const float* z, const uint8_t* mask, int64_t j, float tau, float& zh) {
    const float v = z[j];
    const bool ok = (mask == nullptr || mask[j] != 0) && isfinite(v);
    zh = __fdiv_rn(v, tau);
    return ok;
}

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

__device__ __forceinline__ long long sel_weight(float zh, bool ok, float M) {
    return ok ? __float2ll_rn(expf(zh - M) * kFix) : 0;
}

__global__ void __launch_bounds__(kSelThreads) sel_max_kernel(const float* z, const uint8_t* mask, float tau,
                                                              const SelPart* parts, float* pmax) {
    __shared__ float sm[32];
    const SelPart P = parts[blockIdx.x];
    float m = -INFINITY;
    for (int64_t j = P.begin + threadIdx.x; j < P.end; j += kSelThreads) {
        float zh;
        if (sel_load(z, mask, j, tau, zh)) m = fmaxf(m, zh);
    }
    m = block_max(m, sm);
    if (threadIdx.x == 0) pmax[blockIdx.x] = m;
}

__device__ __forceinline__ float seg_max(const SelSeg& S, const float* pmax) {
    float M = -INFINITY;
    for (int p = 0; p < S.n_parts; ++p) M = fmaxf(M, pmax[S.first_part + p]);
    return M;
}

__global__ void __launch_bounds__(kSelThreads) sel_sum_kernel(const float* z, const uint8_t* mask, float tau,
                                                              const SelSeg* segs, const SelPart* parts,
                                                              const float* pmax, long long* psum, long long* tsum) {
    __shared__ long long sm[32];
    const SelPart P = parts[blockIdx.x];
    const float M = seg_max(segs[P.seg], pmax);
    long long part = 0;
    for (int t = 0; t < kSelTilesPerPart; ++t) {
        const int64_t t0 = P.begin + (int64_t)t * kSelTile;
        long long s = 0;
        if (t0 < P.end && M > -INFINITY) {
#pragma unroll
            for (int i = 0; i < kSelPerThread; ++i) {
                const int64_t j = t0 + i * kSelThreads + threadIdx.x;
                if (j < P.end) {
                    float zh;
                    const bool ok = sel_load(z, mask, j, tau, zh);
                    s += sel_weight(zh, ok, M);
                }
            }
        }
        s = block_sum(s, sm);
        if (threadIdx.x == 0) tsum[(size_t)blockIdx.x * kSelTilesPerPart + t] = s;
        part += s;
    }
    if (threadIdx.x == 0) psum[blockIdx.x] = part;
}

// One CTA per segment.
__global__ void __launch_bounds__(kSelThreads) sel_pick_kernel(const float* z, const uint8_t* mask, float tau,
                                                               const SelSeg* segs, const SelPart* parts,
                                                               const float* pmax, const long long* psum,
                                                               const long long* tsum, uint64_t seed, uint64_t ctr,
                                                               int64_t* out_index, float* out_logp) {
    __shared__ long long s_thr[kSelThreads];
    __shared__ int64_t s_pos;
    __shared__ long long s_rest;
    const int s_id = blockIdx.x;
    const SelSeg S = segs[s_id];
    const float M = seg_max(S, pmax);
    const int tid = threadIdx.x;
    if (tid == 0) {
        long long W = 0;
        for (int p = 0; p < S.n_parts; ++p) W += psum[S.first_part + p];
        int64_t pos = -1;
        long long rest = 0;
        if (W > 0) {
            // u = m 2^-53 from the segment's Philox block, t = floor(u W) exactly
            uint32_t c0 = (uint32_t)ctr, c1 = (uint32_t)(ctr >> 32), c2 = (uint32_t)s_id, c3 = kSelStream;
            philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
            const unsigned long long m = ((unsigned long long)c0 << 21) | (c1 >> 11);
            const unsigned long long lo = m * (unsigned long long)W;
            const unsigned long long hi = __umul64hi(m, (unsigned long long)W);
            long long t = (long long)((hi << 11) | (lo >> 53));
            // part, then tile, whose running sum first exceeds t
            int p = 0;
            while (p < S.n_parts - 1 && t >= psum[S.first_part + p]) t -= psum[S.first_part + p++];
            const int gp = S.first_part + p;
            int k = 0;
            while (k < kSelTilesPerPart - 1 && t >= tsum[(size_t)gp * kSelTilesPerPart + k])
                t -= tsum[(size_t)gp * kSelTilesPerPart + k++];
            pos = parts[gp].begin + (int64_t)k * kSelTile;
            rest = t;
        }
        s_pos = pos;
        s_rest = rest;
        out_logp[s_id] = W > 0 ? 0.f : NAN;
    }
    __syncthreads();
    const int64_t tile0 = s_pos;
    if (tile0 < 0) {
        if (tid == 0) out_index[s_id] = -1;
        return;
    }
    const int64_t seg_end = parts[S.first_part + S.n_parts - 1].end;
    // the tile's logits in order: thread i takes 8 consecutive ones
    const int64_t j0 = tile0 + (int64_t)tid * kSelPerThread;
    long long q[kSelPerThread];
    float zq[kSelPerThread];
    long long own = 0;
#pragma unroll
    for (int i = 0; i < kSelPerThread; ++i) {
        const int64_t j = j0 + i;
        q[i] = 0;
        zq[i] = 0.f;
        if (j < seg_end) {
            const bool ok = sel_load(z, mask, j, tau, zq[i]);
            q[i] = sel_weight(zq[i], ok, M);
        }
        own += q[i];
    }
    s_thr[tid] = own;
    __syncthreads();
    if (tid == 0) {
        // exclusive prefix over the 256 thread sums; the owner of t
        long long t = s_rest;
        int owner = 0;
        while (owner < kSelThreads - 1 && t >= s_thr[owner]) t -= s_thr[owner++];
        s_thr[0] = owner;
        s_rest = t;
    }
    __syncthreads();
    if (tid == (int)s_thr[0]) {
        long long t = s_rest;
        int i = 0;
        while (i < kSelPerThread - 1 && t >= q[i]) t -= q[i++];
        const int64_t j = j0 + i;
        out_index[s_id] = j - S.begin;
        long long W = 0;
        for (int p = 0; p < S.n_parts; ++p) W += psum[S.first_part + p];
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
    sel_max_kernel<<<n_parts, kSelThreads, 0, st>>>(logits, mask, tau, parts, pmax);
    sel_sum_kernel<<<n_parts, kSelThreads, 0, st>>>(logits, mask, tau, segs, parts, pmax, psum, tsum);
    sel_pick_kernel<<<n_seg, kSelThreads, 0, st>>>(logits, mask, tau, segs, parts, pmax, psum, tsum, seed, counter,
                                                   out_index, out_logp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sel_fail(AKMC_ECUDA, std::string("select kernels: ") + cudaGetErrorString(e));
    return AKMC_OK;
}
