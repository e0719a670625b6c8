// Unequal-sized subclustering (Algorithm 2): after feature scaling, L and H are the
// points made of every attribute's lowest and highest value; the segment from L to H is
// cut into m equal pieces whose middles are the landmarks
//     l_i = float(L + ((i + 1/2) / m) (H - L))        (double arithmetic, stored as float)
// and every point joins its nearest landmark.  "Nearest" is the float64 squared distance
// of the peel (ascending attributes, one rounding per operation), the lower landmark index
// on ties.  As in the peel, each point's distances are computed in float32 with the bound
// |d32 - d64| <= eps d32 + 2^-120, eps = (d+4) 2^-23; only when that bound leaves more than
// one landmark in contention are those landmarks' float64 distances computed.
//
// The subclusters are the groups in landmark order with their points in ascending index
// (a stable counting sort: per-tile histograms, a scan over (group, tile), and a stable
// scatter per tile with warp match), groups that nobody joins being left out.
#include "pscl_internal.cuh"

namespace pscl {
namespace {

constexpr int kTile = 1024;                  // points per tile of the counting sort

__global__ void k_landmarks(const double *mn, const double *mx, int d, int m, float *lm)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * d; e += gridDim.x * blockDim.x) {
        const int i = e / d, a = e - i * d;
        const double t = __ddiv_rn((double)i + 0.5, (double)m);
        lm[e] = __double2float_rn(__dadd_rn(mn[a], __dmul_rn(t, __dsub_rn(mx[a], mn[a]))));
    }
}

template <int D>
__device__ __forceinline__ float dist32(const float *x, const float *l, int d)
{
    const int dd = D > 0 ? D : d;
    float acc = 0.0f;
#pragma unroll
    for (int a = 0; a < dd; a++) {
        const float t = __fsub_rn(x[a], l[a]);
        acc = __fmaf_rn(t, t, acc);
    }
    return acc;
}

__device__ __forceinline__ double dist64(const float *x, const float *l, int d)
{
    double s = 0.0;
    for (int a = 0; a < d; a++) {
        const double t = __dsub_rn((double)x[a], (double)l[a]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// Group of every point, and per tile of kTile points the count of every group
// (cnt[g * ntiles + tile]).
template <int D>
__global__ void __launch_bounds__(256) k_group(const float *__restrict__ x, int64_t n, int d,
                                               const float *__restrict__ lm, int m, int32_t *group, uint32_t *cnt,
                                               int ntiles)
{
    extern __shared__ uint32_t hist[];
    for (int g = threadIdx.x; g < m; g += blockDim.x) hist[g] = 0;
    __syncthreads();
    const float eps = (float)(d + 4) * 0x1p-23f;
    const int dd = D > 0 ? D : d;
    const int64_t i0 = (int64_t)blockIdx.x * kTile;
    for (int q = threadIdx.x; q < kTile; q += blockDim.x) {
        const int64_t i = i0 + q;
        if (i >= n) break;
        const float *xi = x + i * dd;
        float xv[D > 0 ? D : 1];
        if (D > 0)
#pragma unroll
            for (int a = 0; a < (D > 0 ? D : 1); a++) xv[a] = __ldg(&xi[a]);
        const float *xp = D > 0 ? xv : xi;
        float best = __int_as_float(0x7f800000);
        int bj = 0;
        for (int j = 0; j < m; j++) {
            const float v = dist32<D>(xp, lm + (size_t)j * dd, dd);
            if (v < best) { best = v; bj = j; }
        }
        // landmarks the float32 bound cannot separate from the best
        const float hi = __fadd_ru(__fmul_ru(best, 1.0f + eps), 0x1p-120f);
        int cand = 0;
        for (int j = 0; j < m && cand < 2; j++) {
            const float v = dist32<D>(xp, lm + (size_t)j * dd, dd);
            if (__fsub_rd(__fmul_rd(v, 1.0f - eps), 0x1p-120f) <= hi) cand++;
        }
        if (cand > 1) {                       // float64, as defined, for those landmarks
            double b64 = 0.0;
            int b = -1;
            for (int j = 0; j < m; j++) {
                const float v = dist32<D>(xp, lm + (size_t)j * dd, dd);
                if (__fsub_rd(__fmul_rd(v, 1.0f - eps), 0x1p-120f) > hi) continue;
                const double w = dist64(xi, lm + (size_t)j * dd, dd);
                if (b < 0 || w < b64) { b64 = w; b = j; }
            }
            bj = b;
        }
        group[i] = bj;
        atomicAdd(&hist[bj], 1u);
    }
    __syncthreads();
    for (int g = threadIdx.x; g < m; g += blockDim.x) cnt[(size_t)g * ntiles + blockIdx.x] = hist[g];
}

// Exclusive scan of cnt (group-major) in place, and every group's total.  One block.
__global__ void __launch_bounds__(1024) k_group_scan(uint32_t *cnt, int64_t len, int ntiles, uint32_t *total)
{
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < len; b0 += 1024) {
        const int64_t e = b0 + threadIdx.x;
        const uint32_t v = e < len ? cnt[e] : 0u;
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) ws[w] = inc;
        __syncthreads();
        if (w == 0) {
            const uint32_t s = ws[lane];
            uint32_t si = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, si, o);
                if (lane >= o) si += u;
            }
            ws[lane] = si - s;
        }
        __syncthreads();
        const uint32_t c = carry;
        if (e < len) cnt[e] = c + ws[w] + inc - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + ws[w] + inc;
        __syncthreads();
    }
    // group totals: the scan at the group's first tile and at the next group's
    for (int g = threadIdx.x; (int64_t)g * ntiles < len; g += blockDim.x) {
        const uint32_t start = cnt[(size_t)g * ntiles];
        const uint32_t end = (int64_t)(g + 1) * ntiles < len ? cnt[(size_t)(g + 1) * ntiles] : carry;
        total[g] = end - start;
    }
}

// Stable scatter of one tile: its points in order, 32 at a time (one warp).
__global__ void __launch_bounds__(32) k_group_scatter(const int32_t *group, int64_t n, const uint32_t *cnt, int m,
                                                      int ntiles, uint32_t *perm)
{
    extern __shared__ uint32_t cur[];
    const int lane = threadIdx.x;
    for (int g = lane; g < m; g += 32) cur[g] = cnt[(size_t)g * ntiles + blockIdx.x];
    __syncwarp();
    const int64_t i0 = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kTile; r += 32) {
        const int64_t i = i0 + r + lane;
        const bool v = i < n;
        const int g = v ? group[i] : -1;
        const uint32_t peers = __match_any_sync(0xffffffffu, g);
        if (v) perm[cur[g] + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
        __syncwarp();
        if (v && lane == __ffs(peers) - 1) cur[g] += __popc(peers);
        __syncwarp();
    }
}

template <int D>
cudaError_t group_launch(const float *x, int64_t n, int d, const float *lm, int m, int32_t *group, uint32_t *cnt,
                         uint32_t *total, uint32_t *perm, cudaStream_t st)
{
    const int ntiles = (int)((n + kTile - 1) / kTile);
    const size_t hs = (size_t)m * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_group<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs);
    if (e != cudaSuccess) return e;
    k_group<D><<<ntiles, 256, hs, st>>>(x, n, d, lm, m, group, cnt, ntiles);
    k_group_scan<<<1, 1024, 0, st>>>(cnt, (int64_t)m * ntiles, ntiles, total);
    e = cudaFuncSetAttribute(k_group_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs);
    if (e != cudaSuccess) return e;
    k_group_scatter<<<ntiles, 32, hs, st>>>(group, n, cnt, m, ntiles, perm);
    return cudaGetLastError();
}

}  // namespace

size_t group_cnt_words(int64_t n, int m) { return (size_t)m * (size_t)((n + kTile - 1) / kTile); }

cudaError_t launch_group_unequal(const float *x, int64_t n, int d, const double *lo, const double *hi, int m,
                                 float *lm, int32_t *group, uint32_t *cnt, uint32_t *total, uint32_t *perm,
                                 cudaStream_t st, KTimer *kt)
{
    kt->begin(st);
    k_landmarks<<<(m * d + 255) / 256, 256, 0, st>>>(lo, hi, d, m, lm);
    cudaError_t e;
    switch (d) {
    case 2: e = group_launch<2>(x, n, d, lm, m, group, cnt, total, perm, st); break;
    case 4: e = group_launch<4>(x, n, d, lm, m, group, cnt, total, perm, st); break;
    case 8: e = group_launch<8>(x, n, d, lm, m, group, cnt, total, perm, st); break;
    case 16: e = group_launch<16>(x, n, d, lm, m, group, cnt, total, perm, st); break;
    case 32: e = group_launch<32>(x, n, d, lm, m, group, cnt, total, perm, st); break;
    case 64: e = group_launch<64>(x, n, d, lm, m, group, cnt, total, perm, st); break;
    default: e = group_launch<0>(x, n, d, lm, m, group, cnt, total, perm, st); break;
    }
    kt->end(PSCL_K_PEEL, st);
    return e;
}

}  // namespace pscl
