// Equal-sized subclustering (Algorithm 1 steps 2-5, repeated on the points left out as
// §II describes): round r builds the landmark L = per-attribute minimum of the
// remaining points, takes the N remaining points nearest to L as subcluster r and
// removes them.
//
// Membership is defined by the float64 distance
//     delta64_i = sum_{j ascending} (double(x_ij) - double(L_j))^2   (one rounding per op)
// with equal distances taken in ascending point index.  Computing delta64 for every
// point would run the whole peel on the slow float64 pipe, so each round works in
// float32 and keeps float64 for a thin band:
//   1. k_peel_dist:     delta32_i by a float32 FMA chain, stored as its bit pattern
//                       (order-preserving for non-negative floats) + a 4096-bin
//                       histogram of bits 31..20; the last block finds the bin holding
//                       the N-th smallest key.
//   2. k_peel_hist1:    a 4096-bin histogram of bits 19..8 inside that bin; the last
//                       block finds the 24-bit prefix [A, B] of the N-th smallest key and
//                       turns it into two float32 cut-offs:
//                       |delta32 - delta64| <= eps*delta32 + ea with eps = (d+4)*2^-23,
//                       ea = 2^-120, so the N-th smallest delta64 lies in
//                       [A(1-eps)-ea, B(1+eps)+ea]; a point whose upper bound lies below
//                       that interval is certainly taken, one whose lower bound lies above
//                       it certainly not.
//   3. k_peel_classify: marks every point in / out / band; band points get delta64
//                       (exactly the definition above) and are listed; the last block
//                       picks the (N - #in) smallest band points by (delta64, position)
//                       with a 96-bit radix select and turns per-block counts into
//                       output offsets.
//   4. k_peel_compact:  stable compaction: taken points go to subcluster r in ascending
//                       index, the others stay in ascending index; the per-attribute
//                       minimum of the points that stay is the next landmark.
// The partition is therefore exactly the float64 definition's, whatever float32 does.
#include "pscl_internal.cuh"

namespace pscl {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kInfBits = 0x7f800000u;

// ------------------------------------------------------------------ block helpers
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan over the block (blockDim.x == kThreads); `total` gets the block sum.
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t &total)
{
    __shared__ uint32_t wsum[kThreads / 32];
    __shared__ uint32_t wtot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < kThreads / 32 ? wsum[lane] : 0;
        uint32_t si = warp_incl_scan(s);
        if (lane < kThreads / 32) wsum[lane] = si - s;
        if (lane == kThreads / 32 - 1) wtot = si;
    }
    __syncthreads();
    uint32_t r = wsum[w] + inc - v;
    total = wtot;
    __syncthreads();
    return r;
}

// In a 4096-bin histogram (global memory), find the bin holding rank `target` (0-based)
// and the rank inside that bin.  Called by a whole block.
__device__ void find_bin(const uint32_t *hist, uint32_t target, uint32_t *bin, uint32_t *rank)
{
    uint32_t tot;
    constexpr int per = kHistBins / kThreads;     // 16 bins per thread
    const int t = threadIdx.x;
    uint32_t loc[per];
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < per; q++) {
        loc[q] = __ldcg(&hist[t * per + q]);
        s += loc[q];
    }
    uint32_t before = block_excl_scan(s, tot);
    if (target >= before && target < before + s) {
        uint32_t c = before;
#pragma unroll
        for (int q = 0; q < per; q++) {
            if (target >= c && target < c + loc[q]) {
                *bin = (uint32_t)(t * per + q);
                *rank = target - c;
            }
            c += loc[q];
        }
    }
}

__device__ __forceinline__ bool last_block(uint32_t *ticket)
{
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// ------------------------------------------------------------------ distances
// float32 distance: t = RN(x - L), acc = RN(t*t + acc) (fused), ascending attributes.
template <int D>
__device__ __forceinline__ float dist32(const float *__restrict__ row, const float *Ls, int d)
{
    float acc = 0.0f;
    if (D > 0 && (D % 4) == 0) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int q = 0; q < D / 4; q++) {
            float4 v = __ldg(&r4[q]);
            float t0 = __fsub_rn(v.x, Ls[4 * q + 0]);
            acc = __fmaf_rn(t0, t0, acc);
            float t1 = __fsub_rn(v.y, Ls[4 * q + 1]);
            acc = __fmaf_rn(t1, t1, acc);
            float t2 = __fsub_rn(v.z, Ls[4 * q + 2]);
            acc = __fmaf_rn(t2, t2, acc);
            float t3 = __fsub_rn(v.w, Ls[4 * q + 3]);
            acc = __fmaf_rn(t3, t3, acc);
        }
    } else {
        const int dd = D > 0 ? D : d;
#pragma unroll 4
        for (int j = 0; j < dd; j++) {
            float t = __fsub_rn(__ldg(&row[j]), Ls[j]);
            acc = __fmaf_rn(t, t, acc);
        }
    }
    return acc;
}

// float64 distance exactly as defined: diff, square, add, each rounded, no fusion.
__device__ double dist64(const float *__restrict__ row, const float *Ls, int d)
{
    double s = 0.0;
    for (int j = 0; j < d; j++) {
        double diff = __dsub_rn((double)row[j], (double)Ls[j]);
        s = __dadd_rn(s, __dmul_rn(diff, diff));
    }
    return s;
}

// ------------------------------------------------------------------ kernels
template <int D>
__global__ void __launch_bounds__(kThreads)
k_peel_dist(const float *__restrict__ x, int d, const uint32_t *__restrict__ idx, uint32_t nr,
            const float *__restrict__ L, uint32_t *__restrict__ key, PeelCtl *ctl, uint32_t target)
{
    __shared__ uint32_t h[kHistBins];
    __shared__ float Ls[D > 0 ? D : kMaxD];
    for (int b = threadIdx.x; b < kHistBins; b += kThreads) h[b] = 0;
    for (int j = threadIdx.x; j < d; j += kThreads) Ls[j] = L[j];
    __syncthreads();
    for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < nr; i += gridDim.x * kThreads) {
        uint32_t row = idx ? idx[i] : i;
        float dl = dist32<D>(x + (size_t)row * d, Ls, d);
        uint32_t k = __float_as_uint(dl);
        key[i] = k;
        atomicAdd(&h[k >> 20], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kHistBins; b += kThreads)
        if (h[b]) atomicAdd(&ctl->hist0[b], h[b]);
    if (!last_block(&ctl->ticket[0])) return;
    find_bin(ctl->hist0, target, &ctl->b0, &ctl->rank0);
    __syncthreads();
    for (int b = threadIdx.x; b < kHistBins; b += kThreads) ctl->hist0[b] = 0;
    if (threadIdx.x == 0) ctl->ticket[0] = 0;
}

__global__ void __launch_bounds__(kThreads)
k_peel_hist1(const uint32_t *__restrict__ key, uint32_t nr, PeelCtl *ctl, int d)
{
    __shared__ uint32_t h[kHistBins];
    for (int b = threadIdx.x; b < kHistBins; b += kThreads) h[b] = 0;
    __syncthreads();
    const uint32_t b0 = ctl->b0;
    for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < nr; i += gridDim.x * kThreads) {
        uint32_t k = key[i];
        if ((k >> 20) == b0) atomicAdd(&h[(k >> 8) & 0xFFFu], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kHistBins; b += kThreads)
        if (h[b]) atomicAdd(&ctl->hist1[b], h[b]);
    if (!last_block(&ctl->ticket[1])) return;
    __shared__ uint32_t b1, r1;
    find_bin(ctl->hist1, ctl->rank0, &b1, &r1);
    __syncthreads();
    for (int b = threadIdx.x; b < kHistBins; b += kThreads) ctl->hist1[b] = 0;
    if (threadIdx.x == 0) {
        uint32_t lo = (b0 << 20) | (b1 << 8);
        uint32_t hi = lo | 0xFFu;
        double A = (double)__uint_as_float(lo), B = (double)__uint_as_float(hi);
        double eps = (double)(d + 4) * 0x1p-23;
        double ea = 0x1p-120;
        double klo = A * (1.0 - eps) - ea;
        double khi = B * (1.0 + eps) + ea;
        double in_thr = (klo - ea) / (1.0 + eps) * (1.0 - 0x1p-40);
        double out_thr = (khi + ea) / (1.0 - eps) * (1.0 + 0x1p-40);
        ctl->in_key = in_thr > 0.0 ? __float_as_uint(__double2float_rd(in_thr)) : 0u;
        ctl->out_key = __float_as_uint(__double2float_ru(out_thr));
        ctl->ticket[1] = 0;
    }
}

// Single-block selection of the `need` smallest (key, pos) pairs of the band list by an
// 8-bit radix select over the 96-bit composite; marks them taken.
__device__ void select_band(const uint64_t *bkey, const uint32_t *bpos, uint32_t nb, uint32_t need,
                            uint8_t *status, uint32_t *blk_cnt)
{
    __shared__ uint32_t h[256];
    __shared__ uint64_t pk;
    __shared__ uint32_t pp, rank;
    if (threadIdx.x == 0) { pk = 0; pp = 0; rank = need - 1; }
    __syncthreads();
    for (int pass = 0; pass < 12; pass++) {
        for (int b = threadIdx.x; b < 256; b += kThreads) h[b] = 0;
        __syncthreads();
        const uint64_t cpk = pk;
        const uint32_t cpp = pp;
        for (uint32_t i = threadIdx.x; i < nb; i += kThreads) {
            uint64_t k = __ldcg(&bkey[i]);
            uint32_t p = __ldcg(&bpos[i]);
            bool match;
            uint32_t digit;
            if (pass < 8) {
                match = pass == 0 || (k >> (64 - 8 * pass)) == (cpk >> (64 - 8 * pass));
                digit = (uint32_t)(k >> (56 - 8 * pass)) & 0xFFu;
            } else {
                int q = pass - 8;
                match = k == cpk && (q == 0 || (p >> (32 - 8 * q)) == (cpp >> (32 - 8 * q)));
                digit = (p >> (24 - 8 * q)) & 0xFFu;
            }
            if (match) atomicAdd(&h[digit], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t c = 0, r = rank;
            for (int b = 0; b < 256; b++) {
                if (r < c + h[b]) {
                    if (pass < 8) pk |= (uint64_t)b << (56 - 8 * pass);
                    else pp |= (uint32_t)b << (24 - 8 * (pass - 8));
                    rank = r - c;
                    break;
                }
                c += h[b];
            }
        }
        __syncthreads();
    }
    const uint64_t K = pk;
    const uint32_t Pp = pp;
    for (uint32_t i = threadIdx.x; i < nb; i += kThreads) {
        uint64_t k = __ldcg(&bkey[i]);
        uint32_t p = __ldcg(&bpos[i]);
        if (k < K || (k == K && p <= Pp)) {
            status[p] = 1;
            atomicAdd(&blk_cnt[p / kBlkItems], 1u);
        }
    }
}

template <int D>
__global__ void __launch_bounds__(kThreads)
k_peel_classify(const float *__restrict__ x, int d, const uint32_t *__restrict__ idx, uint32_t nr,
                const uint32_t *__restrict__ key, const float *__restrict__ L, uint8_t *status,
                uint64_t *band_key, uint32_t *band_pos, uint32_t *blk_cnt, uint32_t *blk_off,
                PeelCtl *ctl, uint32_t N)
{
    __shared__ float Ls[D > 0 ? D : kMaxD];
    uint32_t tot;
    for (int j = threadIdx.x; j < d; j += kThreads) Ls[j] = L[j];
    __syncthreads();
    const uint32_t in_key = ctl->in_key, out_key = ctl->out_key;
    const uint32_t base = blockIdx.x * kBlkItems + threadIdx.x * 4;
    uint32_t n_in = 0;
    uint8_t st[4] = {0, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < 4; q++) {
        uint32_t i = base + q;
        if (i >= nr) break;
        uint32_t k = key[i];
        uint8_t s = k < in_key ? 1 : (k > out_key ? 0 : 2);
        if (s == 2) {
            uint32_t row = idx ? idx[i] : i;
            double dl = dist64(x + (size_t)row * d, Ls, d);
            uint32_t slot = atomicAdd(&ctl->band_count, 1u);
            band_key[slot] = (uint64_t)__double_as_longlong(dl);
            band_pos[slot] = i;
        }
        n_in += s == 1;
        st[q] = s;
    }
    if (base + 3 < nr) {
        *reinterpret_cast<uchar4 *>(&status[base]) = make_uchar4(st[0], st[1], st[2], st[3]);
    } else {
        for (int q = 0; q < 4; q++)
            if (base + q < nr) status[base + q] = st[q];
    }
    block_excl_scan(n_in, tot);
    if (threadIdx.x == 0) blk_cnt[blockIdx.x] = tot;
    if (!last_block(&ctl->ticket[2])) return;

    // ---- last block: settle the band, then per-block output offsets
    __shared__ uint32_t all_in, nb, need;
    const uint32_t nblk = gridDim.x;
    uint32_t s = 0;
    for (uint32_t b = threadIdx.x; b < nblk; b += kThreads) s += __ldcg(&blk_cnt[b]);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ uint32_t ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0;
        for (int w = 0; w < kThreads / 32; w++) a += ws[w];
        all_in = a;
        nb = __ldcg(&ctl->band_count);
        need = N > a ? N - a : 0;
        ctl->n_in = a;
        ctl->need = need;
        if (a > N || need > nb) ctl->error = 1;   // would contradict the error bound
    }
    __syncthreads();
    if (need > 0 && need <= nb) {
        if (need == nb) {
            for (uint32_t i = threadIdx.x; i < nb; i += kThreads) {
                uint32_t p = __ldcg(&band_pos[i]);
                status[p] = 1;
                atomicAdd(&blk_cnt[p / kBlkItems], 1u);
            }
        } else {
            select_band(band_key, band_pos, nb, need, status, blk_cnt);
        }
    }
    __threadfence();
    __syncthreads();
    // exclusive prefix of the per-block taken counts
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < nblk; b0 += kThreads) {
        uint32_t b = b0 + threadIdx.x;
        uint32_t v = b < nblk ? __ldcg(&blk_cnt[b]) : 0;
        uint32_t chunk = 0;
        uint32_t ex = block_excl_scan(v, chunk);
        if (b < nblk) blk_off[b] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += chunk;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ctl->band_count = 0;
        ctl->ticket[2] = 0;
    }
    (void)all_in;
}

template <int D>
__global__ void __launch_bounds__(kThreads)
k_peel_compact(const float *__restrict__ x, int d, const uint32_t *__restrict__ idx, uint32_t nr,
               const uint8_t *__restrict__ status, const uint32_t *__restrict__ blk_off,
               uint32_t *__restrict__ seg_out, uint32_t *__restrict__ idx_out, float *lpart,
               float *L, float *landmark_next, PeelCtl *ctl)
{
    uint32_t tot;
    __shared__ uint32_t smin[D > 0 && D <= 64 ? 1 : kMaxD];
    const uint32_t base = blockIdx.x * kBlkItems + threadIdx.x * 4;
    uint8_t st[4] = {0, 0, 0, 0};
    uint32_t ids[4] = {0, 0, 0, 0};
    uint32_t nsel = 0, nval = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        uint32_t i = base + q;
        if (i < nr) {
            st[q] = status[i];
            ids[q] = idx ? idx[i] : i;
            nsel += st[q] == 1;
            nval++;
        }
    }
    uint32_t pre = block_excl_scan(nsel, tot);
    const uint32_t off = blk_off[blockIdx.x];
    const uint32_t blk_base = blockIdx.x * kBlkItems;
    uint32_t valid_before = base < nr ? base - blk_base : (nr > blk_base ? nr - blk_base : 0);
    uint32_t sel_pos = off + pre;
    uint32_t uns_pos = (blk_base - off) + (valid_before - pre);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (q < (int)nval) {
            if (st[q] == 1) seg_out[sel_pos++] = ids[q];
            else idx_out[uns_pos++] = ids[q];
        }
    }
    // per-attribute minimum of the points that stay (non-negative floats: compare bits)
    if (D > 0 && D <= 64) {
        float mn[D > 0 ? D : 1];
#pragma unroll
        for (int j = 0; j < (D > 0 ? D : 1); j++) mn[j] = __int_as_float(kInfBits);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (q < (int)nval && st[q] != 1) {
                const float *row = x + (size_t)ids[q] * d;
#pragma unroll
                for (int j = 0; j < (D > 0 ? D : 1); j++) mn[j] = fminf(mn[j], __ldg(&row[j]));
            }
        }
        __shared__ float wmin[kThreads / 32][D > 0 && D <= 64 ? D : 1];
#pragma unroll
        for (int j = 0; j < (D > 0 ? D : 1); j++) {
            float v = mn[j];
            for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
            if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5][j] = v;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < d; j += kThreads) {
            float v = wmin[0][j];
            for (int w = 1; w < kThreads / 32; w++) v = fminf(v, wmin[w][j]);
            lpart[(size_t)blockIdx.x * d + j] = v;
        }
    } else {
        for (int j = threadIdx.x; j < d; j += kThreads) smin[j] = kInfBits;
        __syncthreads();
        for (int q = 0; q < 4; q++) {
            if (q < (int)nval && st[q] != 1) {
                const float *row = x + (size_t)ids[q] * d;
                for (int j = 0; j < d; j++) atomicMin(&smin[j], __float_as_uint(row[j]));
            }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < d; j += kThreads)
            lpart[(size_t)blockIdx.x * d + j] = __uint_as_float(smin[j]);
    }
    if (!last_block(&ctl->ticket[3])) return;
    for (int j = threadIdx.x; j < d; j += kThreads) {
        float v = __int_as_float(kInfBits);
        for (uint32_t b = 0; b < gridDim.x; b++) v = fminf(v, __ldcg(&lpart[(size_t)b * d + j]));
        L[j] = v;
        if (landmark_next) landmark_next[j] = v;
    }
    if (threadIdx.x == 0) ctl->ticket[3] = 0;
}

__global__ void k_peel_take_all(const uint32_t *__restrict__ idx, uint32_t nr, uint32_t *seg_out)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x)
        seg_out[i] = idx ? idx[i] : i;
}

template <bool kVec4>
__global__ void k_gather_rows(const float *__restrict__ x, const uint32_t *__restrict__ perm,
                              int64_t n, int d, float *__restrict__ out)
{
    if (kVec4) {
        const int d4 = d / 4;
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        float4 *o4 = reinterpret_cast<float4 *>(out);
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d4;
             e += (int64_t)gridDim.x * blockDim.x) {
            int64_t p = e / d4;
            int q = (int)(e - p * d4);
            o4[e] = __ldg(&x4[(int64_t)perm[p] * d4 + q]);
        }
    } else {
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d;
             e += (int64_t)gridDim.x * blockDim.x) {
            int64_t p = e / d;
            int q = (int)(e - p * d);
            out[e] = __ldg(&x[(int64_t)perm[p] * d + q]);
        }
    }
}

template <int D>
cudaError_t peel_rounds(const PeelBuffers &b, int64_t n, int d, int64_t N, int sm_count,
                        cudaStream_t st, KTimer *kt)
{
    const int64_t S = (n + N - 1) / N;
    cudaMemsetAsync(b.L, 0, sizeof(float) * d, st);            // scaled minima are exactly 0
    if (b.landmarks) cudaMemsetAsync(b.landmarks, 0, sizeof(float) * d, st);
    for (int64_t r = 0; r < S; r++) {
        const uint32_t nr = (uint32_t)(n - r * N);
        const uint32_t *idx_in = r == 0 ? nullptr : b.idx[r & 1];
        uint32_t *idx_out = b.idx[(r + 1) & 1];
        uint32_t *seg_out = b.perm + r * N;
        if ((int64_t)nr <= N) {
            int g = (int)((nr + 255) / 256);
            kt->begin(st);
            k_peel_take_all<<<g, 256, 0, st>>>(idx_in, nr, seg_out);
            kt->end(PSCL_K_PEEL_TAKE, st);
            break;
        }
        int g1 = (int)((nr + kThreads - 1) / kThreads);
        if (g1 > sm_count * 8) g1 = sm_count * 8;
        const int nblk = (int)((nr + kBlkItems - 1) / kBlkItems);
        kt->begin(st);
        k_peel_dist<D><<<g1, kThreads, 0, st>>>(b.x, d, idx_in, nr, b.L, b.key, b.ctl, (uint32_t)(N - 1));
        kt->end(PSCL_K_PEEL_DIST, st);
        kt->begin(st);
        k_peel_hist1<<<g1, kThreads, 0, st>>>(b.key, nr, b.ctl, d);
        kt->end(PSCL_K_PEEL_HIST, st);
        kt->begin(st);
        k_peel_classify<D><<<nblk, kThreads, 0, st>>>(b.x, d, idx_in, nr, b.key, b.L, b.status,
                                                       b.band_key, b.band_pos, b.blk_cnt, b.blk_off,
                                                       b.ctl, (uint32_t)N);
        kt->end(PSCL_K_PEEL_CLASSIFY, st);
        kt->begin(st);
        k_peel_compact<D><<<nblk, kThreads, 0, st>>>(b.x, d, idx_in, nr, b.status, b.blk_off, seg_out,
                                                      idx_out, b.lpart, b.L,
                                                      b.landmarks ? b.landmarks + (r + 1) * d : nullptr,
                                                      b.ctl);
        kt->end(PSCL_K_PEEL_COMPACT, st);
    }
    int64_t work = (d % 4 == 0) ? n * d / 4 : n * d;
    int64_t g = (work + 255) / 256;
    if (g > (int64_t)sm_count * 16) g = (int64_t)sm_count * 16;
    kt->begin(st);
    if (d % 4 == 0)
        k_gather_rows<true><<<(int)g, 256, 0, st>>>(b.x, b.perm, n, d, b.xseg);
    else
        k_gather_rows<false><<<(int)g, 256, 0, st>>>(b.x, b.perm, n, d, b.xseg);
    kt->end(PSCL_K_GATHER, st);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_peel(const PeelBuffers &b, int64_t n, int d, int64_t N, int sm_count,
                        cudaStream_t st, KTimer *kt)
{
    switch (d) {
    case 2: return peel_rounds<2>(b, n, d, N, sm_count, st, kt);
    case 4: return peel_rounds<4>(b, n, d, N, sm_count, st, kt);
    case 8: return peel_rounds<8>(b, n, d, N, sm_count, st, kt);
    case 16: return peel_rounds<16>(b, n, d, N, sm_count, st, kt);
    case 32: return peel_rounds<32>(b, n, d, N, sm_count, st, kt);
    case 64: return peel_rounds<64>(b, n, d, N, sm_count, st, kt);
    default: return peel_rounds<0>(b, n, d, N, sm_count, st, kt);
    }
}

}  // namespace pscl
