// Equal-sized subclustering (Algorithm 1 steps 2-5, repeated on the points left out as
// §II describes): round r builds the landmark L = per-attribute minimum of the
// remaining points, takes the N remaining points nearest to L as subcluster r and
// removes them.
//
// Membership is defined by the float64 distance
//     delta64_i = sum_{j ascending} (double(x_ij) - double(L_j))^2   (one rounding per op)
// with equal distances taken in ascending point index.  Computing delta64 for every
// point would run the peel on the slow float64 pipe, so each round works in float32 and
// keeps float64 for a thin band around the N-th distance:
//   A. delta32_i in float32 (FMA chains, a row's pieces summed across the lanes that read
//      it), kept as its bit pattern (order-preserving for non-negative floats), and a
//      2048-bin histogram of key bits 31..21;
//   B. the bin holding the N-th smallest key, and a 2048-bin histogram of bits 20..10 of
//      the keys inside it: the N-th smallest key lies in a 22-bit prefix [A, B].  The bin
//      is nearly always the previous round's, whose second histogram phase A already
//      built, and then this pass is skipped;
//   C. |delta32 - delta64| <= eps*delta32 + ea with eps = (d+4)*2^-23, ea = 2^-120, so
//      the N-th smallest delta64 lies in [A(1-eps)-ea, B(1+eps)+ea]: a point whose upper
//      bound is below that interval is certainly taken, one whose lower bound is above
//      it certainly not; the few in between form the band;
//   D. the (N - #certain) smallest band points by (delta64, index) are taken, settled in
//      float32, then compensated float32, then float64 for what each step leaves open;
//      taken points go to subcluster r in ascending index and are marked removed.
// The partition is therefore exactly the float64 definition's, whatever float32 does.
//
// Points never move: CTA c owns the index slice [c n/G, (c+1) n/G) in every round and keeps
// the ids of its points left in a list, in ascending order; a removed point gets the key
// 0xFFFFFFFF.  The next landmark needs no pass over the rows.  Before round 0 a counting
// sort lists, per attribute, the point ids by value bucket (buckets are monotone in the
// value) with a live count per bucket that every removal decrements.  The minimum over the
// points left is the smallest value left in the first bucket that still has a point, and
// the buckets in front of it never get one back, so one bucket pointer per attribute only
// moves forward.
//
// All rounds run in one persistent cooperative launch, the phases separated by grid
// barriers (three per round).  Every barrier wait is bounded; a CTA that gives up sets the
// abort flag, every other CTA then leaves at its next wait, and the host sees
// PSCL_ETIMEOUT.
#include <algorithm>

#include "pscl_internal.cuh"

namespace pscl {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kInfBits = 0x7f800000u;
constexpr uint32_t kGone = 0xFFFFFFFFu;       // key of a point removed in an earlier round
constexpr uint32_t kTaken = 0xFFFFFFFEu;      // key of a wide-band point taken this round
constexpr int kBandBins = 4096;               // one-ulp bins over a band's float32 keys
constexpr int kTight = 256;                   // band entries near the cut-off, decided exactly
constexpr int kKeyCache = 4096;               // keys and ids of a slice kept in shared memory, if it fits
constexpr int kPeelScratch = 2 * kHistBins > kBandBins + 7 * kTight ? 2 * kHistBins : kBandBins + 7 * kTight;
constexpr int kBandStage = 4 * 256;           // band entries staged in shared memory (4 per thread)
constexpr int kPeelDynWords = kPeelScratch + 2 * kKeyCache + 2 * kBandStage;
constexpr int kQT = 8;                        // tiles of kThreads items per compaction scan
constexpr int kCB = 16;                       // keys per thread in flight when classifying
constexpr unsigned kSpinLimit = 1u << 25;      // ~1-2 s of polling per barrier at most

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

__device__ uint32_t block_sum(uint32_t v)
{
    uint32_t tot;
    block_excl_scan(v, tot);
    return tot;
}

// In a kHistBins-bin histogram (global memory), find the bin holding rank `target` (0-based)
// and the rank inside that bin.  Called by the whole block; every thread gets the result.
__device__ void find_bin(const uint32_t *hist, uint32_t target, uint32_t &bin, uint32_t &rank)
{
    __shared__ uint32_t sb, sr;
    constexpr int per = kHistBins / kThreads;     // 8 bins per thread
    const int t = threadIdx.x;
    uint32_t loc[per];
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < per; q++) {
        loc[q] = __ldcg(&hist[t * per + q]);
        s += loc[q];
    }
    uint32_t tot;
    uint32_t before = block_excl_scan(s, tot);
    if (target >= before && target < before + s) {
        uint32_t c = before;
#pragma unroll
        for (int q = 0; q < per; q++) {
            if (target >= c && target < c + loc[q]) {
                sb = (uint32_t)(t * per + q);
                sr = target - c;
            }
            c += loc[q];
        }
    }
    __syncthreads();
    bin = sb;
    rank = sr;
    __syncthreads();
}

// Grid-wide barrier with a bounded wait: a monotonic arrival counter (release on
// arrival, acquire while polling), so no reset is needed within a launch.  Returns false
// if the launch is being aborted.
__device__ bool grid_sync(PeelCtl *ctl, uint32_t *flags, unsigned &target)
{
    __shared__ int ok;
    target += gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar_count) : "memory");
        unsigned spins = 0, v;
        for (;;) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&ctl->bar_count) : "memory");
            if ((int)(v - target) >= 0) break;
            if ((++spins & 63) == 0) {
                if (*(volatile unsigned *)&ctl->abort) { good = 0; break; }
                if (spins > kSpinLimit) {
                    atomicExch(&ctl->abort, 1u);
                    atomicOr(&flags[1], 2u);           // timed out
                    good = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// ------------------------------------------------------------------ distances
// float32 distance of one row by one thread (the phase-A path for d not a multiple of 4,
// or below 8): t = RN(x - L), acc = RN(t*t + acc) (fused), ascending attributes.
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

// Compensated float32 distance (h + l, |l| <= ulp(h)/2): each difference is split exactly
// into s + e (TwoSum), s^2 is kept exactly as p + pe (FMA), 2*s*e is folded into the low
// part (e^2 <= 2^-48 s^2 is dropped) and the high parts are summed error-free (TwoSum).
// Its distance to the float64 definition is below eps_ff(d) * (h + l).
__device__ __forceinline__ void dist_ff(const float *__restrict__ row, const float *Ls, int d, float &h, float &l)
{
    float hi = 0.0f, lo = 0.0f;
    for (int j = 0; j < d; j++) {
        const float a = __ldg(&row[j]), b = Ls[j];
        const float s = __fsub_rn(a, b);
        const float bb = __fsub_rn(s, a);                       // TwoSum(a, -b)
        const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(-b, bb));
        const float p = __fmul_rn(s, s);
        const float pe = __fmaf_rn(s, s, -p);
        const float q = __fmaf_rn(__fmul_rn(2.0f, s), e, pe);
        const float t = __fadd_rn(hi, p);                       // TwoSum(hi, p)
        const float bv = __fsub_rn(t, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(p, bv));
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(err, q));
    }
    h = __fadd_rn(hi, lo);                                      // normalise (Fast2Sum)
    l = __fsub_rn(lo, __fsub_rn(h, hi));
}

// Bound on |dff - delta64| / delta64: (d^2 + 8d) u^2 for the compensated sum
// (u = 2^-24) plus (d + 2) 2^-53 for the float64 one, with a factor two of margin.
__device__ __forceinline__ float eps_ff(int d)
{
    return (float)((double)d * d + 8.0 * d + 1.0) * 0x1p-47f;
}

// Thresholds of phase C from the 22-bit key prefix [A, B] of the N-th smallest key.
// With eps = (d+4) 2^-23 and ea = 2^-120 the N-th smallest delta64 lies in
// [A(1-eps) - ea, B(1+eps) + ea]; a point is certainly in if delta32 (1+eps) + ea is below
// that interval, which holds for delta32 < A(1-2eps) - 2ea, and certainly out if
// delta32 (1-eps) - ea is above it, which holds for delta32 > B(1+3eps) + 3ea.  Both
// cut-offs are evaluated in float32 rounded towards the safe side.
__device__ void band_cutoffs_key(uint32_t lo, uint32_t hi, int d, uint32_t &in_key, uint32_t &out_key)
{
    const float A = __uint_as_float(lo), B = __uint_as_float(hi);
    const float eps = (float)(d + 4) * 0x1p-23f;
    const float in_thr = __fsub_rd(__fmul_rd(A, __fsub_rd(1.0f, 2.0f * eps)), 0x1p-119f);
    const float out_thr = __fadd_ru(__fmul_ru(B, __fadd_ru(1.0f, 3.0f * eps)), 0x1.8p-119f);
    in_key = in_thr > 0.0f ? __float_as_uint(in_thr) : 0u;
    out_key = __float_as_uint(out_thr);
}

__device__ void band_cutoffs(uint32_t b0, uint32_t b1, int d, uint32_t &in_key, uint32_t &out_key)
{
    const uint32_t lo = (b0 << 21) | (b1 << 10);
    band_cutoffs_key(lo, lo | 0x3FFu, d, in_key, out_key);
}

// Single-block radix select (8-bit digits over the 96-bit (key, pos) composite) of the
// `need`-th smallest band entry in global memory; for bands too large for shared memory.
__device__ void select_band_global(const uint64_t *bkey, const uint32_t *bpos, uint32_t nb, uint32_t need,
                                   uint64_t &K, uint32_t &Pp)
{
    __shared__ uint32_t h[256];
    __shared__ uint64_t pk;
    __shared__ uint32_t pp, rank;
    if (threadIdx.x == 0) { pk = 0; pp = 0; rank = need - 1; }
    __syncthreads();
    for (int pass = 0; pass < 12; pass++) {
        h[threadIdx.x] = 0;
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
        const uint32_t v = h[threadIdx.x];
        uint32_t tot;
        const uint32_t before = block_excl_scan(v, tot);
        const uint32_t r = rank;
        __syncthreads();
        if (r >= before && r < before + v) {
            if (pass < 8) pk = cpk | ((uint64_t)threadIdx.x << (56 - 8 * pass));
            else pp = cpp | ((uint32_t)threadIdx.x << (24 - 8 * (pass - 8)));
            rank = r - before;
        }
        __syncthreads();
    }
    K = pk;
    Pp = pp;
    __syncthreads();
}

// The same selection in three passes when the band's keys spread: the smallest and
// largest key give the bits all keys share; an 11-bit histogram of the next bits finds
// the digit of the need-th entry; that digit's entries (at most kSelList) are gathered in
// shared memory and ranked there by (key, position).  Returns false, with nothing
// decided, when all keys are equal or the digit holds more entries: the caller then runs
// select_band_global.  scratch: 2048 + 3 kSelList words of shared memory.
constexpr int kSelBins = 2048;
constexpr int kSelList = 1024;
constexpr int kSelBatch = 8;
__device__ bool select_band_fast(const uint64_t *bkey, const uint32_t *bpos, uint32_t nb, uint32_t need,
                                 uint32_t *scratch, uint64_t &K, uint32_t &Pp)
{
    __shared__ unsigned long long s_mn[kThreads / 32], s_mx[kThreads / 32];
    __shared__ uint32_t s_bin, s_rank, s_cnt, s_hit;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t *h = scratch;
    uint64_t *lk = reinterpret_cast<uint64_t *>(scratch + kSelBins);      // 8-byte aligned: kSelBins is even
    uint32_t *lp = scratch + kSelBins + 2 * kSelList;
    // pass 1: smallest and largest key
    // every pass keeps kSelBatch loads per thread in flight: one CTA reads the whole band
    unsigned long long mn = ~0ull, mx = 0ull;
    for (uint32_t i0 = t; i0 < nb; i0 += kSelBatch * kThreads) {
        unsigned long long kk[kSelBatch];
#pragma unroll
        for (int u = 0; u < kSelBatch; u++) {
            const uint32_t i = i0 + u * kThreads;
            kk[u] = i < nb ? __ldcg(&bkey[i]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kSelBatch; u++) {
            if (i0 + u * kThreads < nb) {
                mn = min(mn, kk[u]);
                mx = max(mx, kk[u]);
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        s_mn[w] = mn;
        s_mx[w] = mx;
    }
    for (int b = t; b < kSelBins; b += kThreads) h[b] = 0;
    __syncthreads();
    mn = s_mn[0];
    mx = s_mx[0];
#pragma unroll
    for (int q = 1; q < kThreads / 32; q++) {
        mn = min(mn, (unsigned long long)s_mn[q]);
        mx = max(mx, (unsigned long long)s_mx[q]);
    }
    if (mn == mx) return false;                          // uniform across the block
    const int hb = 63 - __clzll((long long)(mn ^ mx));   // highest bit where keys differ
    const int sh = hb >= 10 ? hb - 10 : 0;               // digit = bits [sh, hb]
    // pass 2: histogram of the digit (the bits above hb are common to all keys)
    for (uint32_t i0 = t; i0 < nb; i0 += kSelBatch * kThreads) {
        unsigned long long kk[kSelBatch];
#pragma unroll
        for (int u = 0; u < kSelBatch; u++) {
            const uint32_t i = i0 + u * kThreads;
            kk[u] = i < nb ? __ldcg(&bkey[i]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kSelBatch; u++)
            if (i0 + u * kThreads < nb) atomicAdd(&h[(uint32_t)(kk[u] >> sh) & (kSelBins - 1)], 1u);
    }
    __syncthreads();
    {
        constexpr int per = kSelBins / kThreads;
        uint32_t loc = 0;
#pragma unroll
        for (int q = 0; q < per; q++) loc += h[t * per + q];
        uint32_t tot;
        const uint32_t before = block_excl_scan(loc, tot);
        const uint32_t target = need - 1;
        if (target >= before && target < before + loc) {
            uint32_t cc = before;
            for (int q = 0; q < per; q++) {
                const uint32_t v = h[t * per + q];
                if (target >= cc && target < cc + v) {
                    s_bin = (uint32_t)(t * per + q);
                    s_rank = target - cc;
                    s_cnt = v;
                }
                cc += v;
            }
        }
        if (t == 0) s_hit = 0;
    }
    __syncthreads();
    const uint32_t bin = s_bin, rank = s_rank, cnt = s_cnt;
    if (cnt > (uint32_t)kSelList) return false;          // uniform across the block
    // pass 3: the digit's entries, then their rank by (key, position)
    for (uint32_t i0 = t; i0 < nb; i0 += kSelBatch * kThreads) {
        unsigned long long kk[kSelBatch];
#pragma unroll
        for (int u = 0; u < kSelBatch; u++) {
            const uint32_t i = i0 + u * kThreads;
            kk[u] = i < nb ? __ldcg(&bkey[i]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kSelBatch; u++) {
            const uint32_t i = i0 + u * kThreads;
            if (i < nb && ((uint32_t)(kk[u] >> sh) & (kSelBins - 1)) == bin) {
                const uint32_t slot = atomicAdd(&s_hit, 1u);
                lk[slot] = kk[u];
                lp[slot] = __ldcg(&bpos[i]);
            }
        }
    }
    __syncthreads();
    for (uint32_t q = t; q < cnt; q += kThreads) {
        const uint64_t kq = lk[q];
        const uint32_t pq = lp[q];
        uint32_t rk = 0;
        for (uint32_t o = 0; o < cnt; o++) rk += (lk[o] < kq) || (lk[o] == kq && lp[o] < pq);
        if (rk == rank) {
            s_mn[0] = kq;
            s_hit = pq;
        }
    }
    __syncthreads();
    K = s_mn[0];
    Pp = s_hit;
    __syncthreads();
    return true;
}

// Exclusive scans of two values over the block in one pass (blockDim.x == kThreads).
__device__ void block_excl_scan2(uint32_t v0, uint32_t v1, uint32_t &e0, uint32_t &e1, uint32_t &t0,
                                 uint32_t &t1)
{
    constexpr int W = kThreads / 32;
    __shared__ uint32_t ws0[W], ws1[W], wt[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t i0 = warp_incl_scan(v0), i1 = warp_incl_scan(v1);
    if (lane == 31) {
        ws0[w] = i0;
        ws1[w] = i1;
    }
    __syncthreads();
    if (w == 0) {
        const uint32_t a = lane < W ? ws0[lane] : 0u, b = lane < W ? ws1[lane] : 0u;
        const uint32_t ia = warp_incl_scan(a), ib = warp_incl_scan(b);
        if (lane < W) {
            ws0[lane] = ia - a;
            ws1[lane] = ib - b;
        }
        if (lane == W - 1) {
            wt[0] = ia;
            wt[1] = ib;
        }
    }
    __syncthreads();
    e0 = ws0[w] + i0 - v0;
    e1 = ws1[w] + i1 - v1;
    t0 = wt[0];
    t1 = wt[1];
    __syncthreads();
}

__device__ __forceinline__ uint32_t warp_min(uint32_t v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The bin of rank `target` (0-based) of histogram h0 and the rank inside it; when hg (the
// second-digit histogram inside bin `guess`) is given and `guess` is that bin, also the
// bin of that rank in hg (hit).  Both histograms are read and scanned in one pass.
__device__ void find_bins(const uint32_t *h0, const uint32_t *hg, uint32_t guess, uint32_t target,
                          uint32_t &b0, uint32_t &r0, uint32_t &b1, uint32_t &r1, bool &hit)
{
    __shared__ uint32_t sb0, sr0, sb1, sr1;
    constexpr int per = kHistBins / kThreads;       // 8 bins per thread
    static_assert(per == 8, "two uint4 loads per thread");
    const int t = threadIdx.x;
    uint32_t l0[per], l1[per];
    {
        const uint4 *p = reinterpret_cast<const uint4 *>(h0 + t * per);
        const uint4 u = __ldcg(p), v = __ldcg(p + 1);
        l0[0] = u.x; l0[1] = u.y; l0[2] = u.z; l0[3] = u.w;
        l0[4] = v.x; l0[5] = v.y; l0[6] = v.z; l0[7] = v.w;
    }
    if (hg) {
        const uint4 *p = reinterpret_cast<const uint4 *>(hg + t * per);
        const uint4 u = __ldcg(p), v = __ldcg(p + 1);
        l1[0] = u.x; l1[1] = u.y; l1[2] = u.z; l1[3] = u.w;
        l1[4] = v.x; l1[5] = v.y; l1[6] = v.z; l1[7] = v.w;
    } else {
#pragma unroll
        for (int q = 0; q < per; q++) l1[q] = 0;
    }
    uint32_t s0 = 0, s1 = 0;
#pragma unroll
    for (int q = 0; q < per; q++) {
        s0 += l0[q];
        s1 += l1[q];
    }
    uint32_t e0, e1, tot0, tot1;
    block_excl_scan2(s0, s1, e0, e1, tot0, tot1);
    if (target >= e0 && target < e0 + s0) {
        uint32_t cc = e0;
#pragma unroll
        for (int q = 0; q < per; q++) {
            if (target >= cc && target < cc + l0[q]) {
                sb0 = (uint32_t)(t * per + q);
                sr0 = target - cc;
            }
            cc += l0[q];
        }
    }
    __syncthreads();
    b0 = sb0;
    r0 = sr0;
    hit = hg != nullptr && b0 == guess;
    if (hit) {
        if (r0 >= e1 && r0 < e1 + s1) {
            uint32_t cc = e1;
#pragma unroll
            for (int q = 0; q < per; q++) {
                if (r0 >= cc && r0 < cc + l1[q]) {
                    sb1 = (uint32_t)(t * per + q);
                    sr1 = r0 - cc;
                }
                cc += l1[q];
            }
        }
        __syncthreads();
        b1 = sb1;
        r1 = sr1;
    }
    __syncthreads();
}

// Splits the n_in ids of a CTA's list (id_of(q) for position q), keeping their order, into
// those with pred(position, id), written to sel[0..) with on_sel(id) called for each, and the
// rest, written to keep[0..) when `keep` is given.  `keep` may be the list being read (in
// shared memory): a tile's ids are all read before any of its kept ids is written, and those
// land at or below the tile's own positions.  Returns how many were selected (to every
// thread).
template <class IdOf, class Pred, class OnSel>
__device__ uint32_t compact_list(IdOf id_of, uint32_t n_in, uint32_t *sel, uint32_t *keep, Pred pred, OnSel on_sel)
{
    constexpr int W = kThreads / 32;
    constexpr int PER = kQT * W / 32;
    static_assert(PER * 32 == kQT * W, "one warp scans the tile counts");
    __shared__ uint32_t woff_s[kQT * W + 1], woff_k[kQT * W + 1];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t done_s = 0, done_k = 0;
    // item (q, t) of a chunk is preceded by the earlier tiles, the earlier warps of its tile
    // and the lower lanes of its warp
    for (uint32_t cb = 0; cb < n_in; cb += kQT * kThreads) {
        uint32_t ids[kQT], vl = 0, tk = 0;
#pragma unroll
        for (int q = 0; q < kQT; q++) {
            const uint32_t qi = cb + q * kThreads + t;
            const bool v = qi < n_in;
            ids[q] = v ? id_of(qi) : 0u;
            vl |= (uint32_t)v << q;
        }
#pragma unroll
        for (int q = 0; q < kQT; q++) tk |= (uint32_t)(((vl >> q) & 1u) && pred(cb + q * kThreads + t, ids[q])) << q;
        uint32_t bt[kQT], bv[kQT];
#pragma unroll
        for (int q = 0; q < kQT; q++) {
            bt[q] = __ballot_sync(0xffffffffu, (tk >> q) & 1u);
            bv[q] = __ballot_sync(0xffffffffu, (vl >> q) & 1u);
            if (lane == 0) {
                woff_s[q * W + w] = __popc(bt[q]);
                woff_k[q * W + w] = __popc(bv[q] & ~bt[q]);
            }
        }
        __syncthreads();
        if (w == 0) {
            uint32_t vs[PER], vk[PER], ss = 0, sk = 0;
#pragma unroll
            for (int e = 0; e < PER; e++) {
                vs[e] = woff_s[lane * PER + e];
                vk[e] = woff_k[lane * PER + e];
                ss += vs[e];
                sk += vk[e];
            }
            const uint32_t is = warp_incl_scan(ss), ik = warp_incl_scan(sk);
            uint32_t es = is - ss, ek = ik - sk;
#pragma unroll
            for (int e = 0; e < PER; e++) {
                woff_s[lane * PER + e] = es;
                woff_k[lane * PER + e] = ek;
                es += vs[e];
                ek += vk[e];
            }
            if (lane == 31) {
                woff_s[kQT * W] = is;
                woff_k[kQT * W] = ik;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kQT; q++) {
            if ((tk >> q) & 1u) {
                sel[done_s + woff_s[q * W + w] + __popc(bt[q] & lt)] = ids[q];
                on_sel(ids[q]);
            } else if (((vl >> q) & 1u) && keep) {
                keep[done_k + woff_k[q * W + w] + __popc(bv[q] & ~bt[q] & lt)] = ids[q];
            }
        }
        done_s += woff_s[kQT * W];
        done_k += woff_k[kQT * W];
        __syncthreads();
    }
    return done_s;
}

// Bucket of a scaled value (in [0, 1]) among nb equal buckets: monotone in the value.
__device__ __forceinline__ uint32_t bucket_of(float v, uint32_t nb)
{
    v = fminf(fmaxf(v, 0.0f), 1.0f);
    const uint32_t b = __float2uint_rz(v * (float)nb);
    return b < nb ? b : nb - 1u;
}

// The round's selection: a point with key k is taken if k < lo, if it is a wide-band point
// marked kTaken, or if lo <= k <= tout and the tight set lists it as taken.
// Phase C over a slice's keys (key_at(position)): counts those below in_key (certainly
// taken) and hands those in [in_key, out_key] to to_band(position, key); CB keys per
// thread are read at once.
template <int CB, class KeyAt, class ToBand>
__device__ __forceinline__ uint32_t classify_keys(uint32_t n_live, uint32_t in_key, uint32_t out_key, KeyAt key_at,
                                                  ToBand to_band)
{
    uint32_t n_in = 0;
    for (uint32_t q0 = threadIdx.x; q0 < n_live; q0 += CB * kThreads) {
        uint32_t kk[CB];
#pragma unroll
        for (int q = 0; q < CB; q++) {
            const uint32_t qi = q0 + q * kThreads;
            kk[q] = qi < n_live ? key_at(qi) : kGone;       // past the end: above out_key
        }
#pragma unroll
        for (int q = 0; q < CB; q++) {
            if (kk[q] < in_key) n_in++;
            else if (kk[q] <= out_key) to_band(q0 + q * kThreads, kk[q]);
        }
    }
    return n_in;
}

struct Rule {
    uint32_t lo, tout, nt;
    const uint32_t *tpos, *tcls;
};

__device__ __forceinline__ bool taken(const Rule &R, uint32_t k, uint32_t id)
{
    if (k < R.lo || k == kTaken) return true;
    if (k > R.tout) return false;
    for (uint32_t o = 0; o < R.nt; o++)
        if (R.tpos[o] == id) return R.tcls[o] != 0;
    return false;
}

// A removed point leaves the live count of its bucket in every attribute.
template <int D>
__device__ __forceinline__ void drop_buckets(const float *__restrict__ x, int d, uint32_t id, uint4 *bcs, uint32_t nbk)
{
    const float *row = x + (size_t)id * d;
    if (D > 0 && D % 4 == 0) {
        float v[D > 0 ? D : 1];
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int q = 0; q < D / 4; q++) {
            const float4 u = __ldg(&r4[q]);
            v[4 * q + 0] = u.x;
            v[4 * q + 1] = u.y;
            v[4 * q + 2] = u.z;
            v[4 * q + 3] = u.w;
        }
#pragma unroll
        for (int j = 0; j < D; j++) atomicSub(&bcs[(size_t)j * nbk + bucket_of(v[j], nbk)].x, 1u);
    } else {
        for (int j = 0; j < d; j++) atomicSub(&bcs[(size_t)j * nbk + bucket_of(__ldg(&row[j]), nbk)].x, 1u);
    }
}

// ------------------------------------------------------------------ the kernel
struct PeelArgs {
    const float *x;
    int d;
    int64_t n, N, S;
    uint32_t *key;               // n: this round's float32 key per point; kGone once removed
    uint32_t *ord;               // d x ord_ld: point ids by value bucket, per attribute
    uint32_t *bcnt;              // d x nbk: bucket counts, then cursors (zeroed before)
    uint4 *bcs;                  // d x nbk: (points left, first entry, end entry, 0)
    uint32_t *lidx;              // 2 x n: per CTA slice, the ids of its points left
    uint32_t *kpos;              // n: per CTA slice, this round's keys by list position (!kc)
    int64_t ord_ld;
    uint32_t nbk;
    uint64_t *band_key;          // float64 distance bits (wide bands only)
    uint32_t *band_k32;          // float32 keys of the band
    uint32_t *band_pos;          // point ids of the band
    uint32_t *perm;
    float *landmarks;            // S x d or NULL
    PeelCtl *ctl;
    uint32_t *flags;             // job flags: [1] |= 1 bound violated, 2 barrier timed out
};

// rows a thread keeps in flight at once (64 floats of rows at most)
template <int D>
__host__ __device__ constexpr int kPeelBatch()
{
    return D <= 0 ? 1 : (D >= 64 ? 1 : (64 / D > 4 ? 4 : 64 / D));
}

// Phase A reads a row with P = min(D/4, 32) lanes, one float4 each (F per lane when D > 128),
// so that one warp load covers 32/P whole rows instead of one 16-byte piece of 32 rows: the
// L1 then looks up 8 lines per load at D = 16 instead of 32.  Each lane sums its part of P
// rows (fused, ascending attributes) and a butterfly over the P lanes leaves every lane the
// whole sum of one row.  Every squared difference passes through at most D/P + log2 P
// roundings, fewer than the d of the recursive sum that the phase-C error bound allows.
template <int D>
__host__ __device__ constexpr bool kCoopRows()
{
    return D >= 8 && D % 4 == 0;
}

template <int D>
__host__ __device__ constexpr int kCoopLanes()
{
    return D / 4 < 32 ? D / 4 : 32;
}

// 32-row warp chunks a thread keeps in flight: about 16 float4 loads per lane
template <int D>
__host__ __device__ constexpr int kCoopBatch()
{
    return 16 / (D / 4) >= 4 ? 4 : (16 / (D / 4) >= 1 ? 16 / (D / 4) : 1);
}

// Phase A with P lanes per row (see kCoopRows): every live point's float32 key, stored by id
// and by list position (shared memory when kc) and counted in the first histogram and, when
// a bin was guessed, in the second.  Out of line, so that the register allocation of the
// kernel's other phases does not carry its loads in flight.
template <int D>
__device__ __noinline__ void coop_keys(const float *__restrict__ x, const float *Ls, uint32_t n_live, uint32_t s0,
                                       bool round0, bool kc, const uint32_t *sid, const uint32_t *glin, uint32_t *key,
                                       uint32_t *skey, uint32_t *kpos, uint32_t *sh, uint32_t *gh, uint32_t guess)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const bool have_guess = guess != kGone;
    auto LID = [&](uint32_t q) -> uint32_t { return round0 ? s0 + q : kc ? sid[q] : __ldcg(&glin[q]); };
    auto key_out = [&](bool live, uint32_t pos, uint32_t id, uint32_t k) {
        if (live) {
            key[id] = k;
            if (kc) skey[pos] = k;
            else kpos[s0 + pos] = k;
        }
        const uint32_t b = live ? (k >> 21) : kGone;
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        if (live && lane == __ffs(peers) - 1) atomicAdd(&sh[b], (uint32_t)__popc(peers));
        if (have_guess) {
            const uint32_t g2 = live && (k >> 21) == guess ? (k >> 10) & (kHistBins - 1) : kGone;
            const uint32_t pg = __match_any_sync(0xffffffffu, g2);
            if (g2 != kGone && lane == __ffs(pg) - 1) atomicAdd(&gh[g2], (uint32_t)__popc(pg));
        }
    };
    constexpr int P = kCoopLanes<D>();                 // lanes per row
    constexpr int F = D / (4 * P);                     // float4 per lane and row
    constexpr int RW = 32 / P;                         // rows per warp load
    constexpr int BC = kCoopBatch<D>();
    static_assert((P & (P - 1)) == 0 && P >= 2, "lanes per row: a power of two");
    const int g = lane / P, sl = lane % P;
    float4 Lq[F];
#pragma unroll
    for (int f = 0; f < F; f++) {
        const int j = 4 * (sl + P * f);
        Lq[f] = make_float4(Ls[j], Ls[j + 1], Ls[j + 2], Ls[j + 3]);
    }
#pragma unroll 1
    for (uint32_t base = 0; base < n_live; base += BC * kThreads) {
        // chunk q of this warp: list positions cb + [0, 32); lane i fetches the id of
        // position cb + i, and row u of its group is position cb + u*RW + g.  Past the
        // end the id is the slice's first row (read again, an L1 hit).
        uint32_t myid[BC];
#pragma unroll
        for (int q = 0; q < BC; q++) {
            const uint32_t pos = base + q * kThreads + w * 32 + lane;
            myid[q] = pos < n_live ? LID(pos) : s0;
        }
        float4 v[BC][P][F];
#pragma unroll
        for (int q = 0; q < BC; q++)
#pragma unroll
            for (int u = 0; u < P; u++) {
                const uint32_t id = __shfl_sync(0xffffffffu, myid[q], u * RW + g);
                const float4 *r4 = reinterpret_cast<const float4 *>(x + (size_t)id * D) + sl;
#pragma unroll
                for (int f = 0; f < F; f++) v[q][u][f] = __ldg(r4 + P * f);
            }
#pragma unroll
        for (int q = 0; q < BC; q++) {
            float ps[P];
#pragma unroll
            for (int u = 0; u < P; u++) {
                float acc = 0.0f;
#pragma unroll
                for (int f = 0; f < F; f++) {
                    const float t0 = __fsub_rn(v[q][u][f].x, Lq[f].x);
                    acc = __fmaf_rn(t0, t0, acc);
                    const float t1 = __fsub_rn(v[q][u][f].y, Lq[f].y);
                    acc = __fmaf_rn(t1, t1, acc);
                    const float t2 = __fsub_rn(v[q][u][f].z, Lq[f].z);
                    acc = __fmaf_rn(t2, t2, acc);
                    const float t3 = __fsub_rn(v[q][u][f].w, Lq[f].w);
                    acc = __fmaf_rn(t3, t3, acc);
                }
                ps[u] = acc;
            }
            // butterfly: after the round with mask m a lane keeps the half of rows
            // whose index has its lane bit m; at the end ps[0] is row sl's sum
            constexpr int LP = P >= 32 ? 5 : P >= 16 ? 4 : P >= 8 ? 3 : P >= 4 ? 2 : 1;
#pragma unroll
            for (int lv = 1; lv <= LP; lv++) {
                const int m = P >> lv;
                const bool up = (sl & m) != 0;
#pragma unroll
                for (int i = 0; i < m; i++) {
                    const float keep = up ? ps[i + m] : ps[i];
                    const float send = up ? ps[i] : ps[i + m];
                    ps[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, m));
                }
            }
            const uint32_t src = (uint32_t)(sl * RW + g);
            const uint32_t pos = base + q * kThreads + w * 32 + src;
            const uint32_t id = __shfl_sync(0xffffffffu, myid[q], src);
            key_out(pos < n_live, pos, id, __float_as_uint(ps[0]));
        }
    }
}

template <int D>
__global__ void __launch_bounds__(kThreads) k_peel(PeelArgs a)
{
    constexpr int B = kPeelBatch<D>();
    constexpr int W = kThreads / 32;
    // dynamic shared memory: [first histogram | guessed second-digit histogram] in phase A;
    // in phase D the band's one-ulp bins and, kept to the end of the round, the tight set
    extern __shared__ __align__(16) uint32_t dyn[];
    uint32_t *sh = dyn;
    uint32_t *gh = dyn + kHistBins;
    uint32_t *hb = dyn;
    uint32_t *tpos = dyn + kBandBins;
    uint32_t *tcls = tpos + kTight;                    // 1 taken, 0 not
    float *th = reinterpret_cast<float *>(tcls + kTight);
    float *tl = th + kTight;
    uint32_t *tamb = reinterpret_cast<uint32_t *>(tl + kTight);    // undecided tight entries
    unsigned long long *td = reinterpret_cast<unsigned long long *>(tamb + kTight);
    uint32_t *skey = dyn + kPeelScratch;               // keys by list position (kc)
    uint32_t *sid = skey + kKeyCache;                  // ids by list position (kc)
    uint32_t *s_bk = sid + kKeyCache;                  // the band's keys and ids (nb <= kBandStage)
    uint32_t *s_bp = s_bk + kBandStage;
    __shared__ float Ls[D > 0 ? D : kMaxD];
    __shared__ uint32_t s_in_key, s_out_key, s_nt, s_na, s_v, s_t32, s_st, s_en;
    __shared__ uint32_t red_a[W], red_b[W];
    PeelCtl *ctl = a.ctl;
    const int d = a.d;
    const uint32_t n = (uint32_t)a.n, N = (uint32_t)a.N, nbk = a.nbk;
    const int t = threadIdx.x;
    const int lane = t & 31, w = t >> 5;
    const unsigned G = gridDim.x, c = blockIdx.x;
    // With 16 CTAs or more, the last Gl CTAs own no points and only build landmarks, which
    // then overlaps with the others' compaction; otherwise every CTA does both.
    const int Gl = G >= 16 ? min(d, (int)(G / 8)) : 0;
    const unsigned Gs = G - (unsigned)Gl;
    const uint32_t s0 = c < Gs ? (uint32_t)((uint64_t)c * n / Gs) : n;
    const uint32_t s1 = c < Gs ? (uint32_t)((uint64_t)(c + 1) * n / Gs) : n;
    const int lm_first = Gl ? (int)c - (int)Gs : (int)(G - 1 - c);
    const int lm_step = Gl ? Gl : (int)G;
    uint32_t n_live = s1 - s0;           // points of the slice left (ids in lidx after round 0)
    const bool kc = s1 - s0 <= (uint32_t)kKeyCache;   // the round's keys stay in shared memory
    unsigned gen = 0;

    // ---- before round 0: per attribute, the point ids by value bucket (counting sort)
    {
        const uint64_t stride = (uint64_t)G * kThreads;
        const uint32_t si = (uint32_t)(stride / (uint64_t)d), sj = (uint32_t)(stride % (uint64_t)d);
        const uint64_t e0 = (uint64_t)c * kThreads + t;
        for (int pass = 0; pass < 2; pass++) {
            uint32_t i = (uint32_t)(e0 / (uint64_t)d), j = (uint32_t)(e0 % (uint64_t)d);
            while (i < n) {
                const float v = __ldg(&a.x[(size_t)i * d + j]);
                uint32_t *cnt = &a.bcnt[(size_t)j * nbk + bucket_of(v, nbk)];
                if (pass == 0) atomicAdd(cnt, 1u);
                else a.ord[(size_t)j * a.ord_ld + atomicAdd(cnt, 1u)] = i;
                i += si;
                j += sj;
                if (j >= (uint32_t)d) {
                    j -= (uint32_t)d;
                    i++;
                }
            }
            if (!grid_sync(ctl, a.flags, gen)) return;
            if (pass == 1) break;
            // exclusive scan of each attribute's counts in place: they become the cursors
            for (int jj = (int)c; jj < d; jj += (int)G) {
                uint32_t *cj = a.bcnt + (size_t)jj * nbk;
                uint32_t run = 0;
                for (uint32_t b0 = 0; b0 < nbk; b0 += 16 * kThreads) {
                    uint4 *p4 = reinterpret_cast<uint4 *>(cj + b0 + 16 * t);
                    uint32_t v[16];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const uint4 u = __ldcg(p4 + q);
                        v[4 * q + 0] = u.x;
                        v[4 * q + 1] = u.y;
                        v[4 * q + 2] = u.z;
                        v[4 * q + 3] = u.w;
                    }
                    uint32_t s = 0;
#pragma unroll
                    for (int q = 0; q < 16; q++) s += v[q];
                    uint32_t tot;
                    uint32_t acc = run + block_excl_scan(s, tot);
                    uint4 *bs = a.bcs + (size_t)jj * nbk + b0 + 16 * t;
#pragma unroll
                    for (int q = 0; q < 16; q++) {
                        const uint32_t cur = v[q];
                        bs[q] = make_uint4(cur, acc, acc + cur, 0u);
                        v[q] = acc;
                        acc += cur;
                    }
#pragma unroll
                    for (int q = 0; q < 4; q++) p4[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    run += tot;
                }
            }
            if (!grid_sync(ctl, a.flags, gen)) return;
        }
    }

    uint32_t guess = kGone;            // first digit of the previous round's N-th key
    for (int64_t r = 0; r < a.S; r++) {
        const uint32_t nr = (uint32_t)(a.n - r * a.N);
        const int par = (int)(r & 1);
        uint32_t *seg_out = a.perm + r * a.N;
        if (c == 0 && a.landmarks)
            for (int j = t; j < d; j += kThreads)
                a.landmarks[r * d + j] = __uint_as_float(__ldcg(&ctl->Lbits[par][j]));
        // the slice's list of ids left: the slice itself in round 0, then in shared memory
        // when it fits the key cache (compacted there in place), else in global memory
        const uint32_t *glin = a.lidx + (size_t)par * n + s0;
        auto LID = [&](uint32_t q) -> uint32_t { return r == 0 ? s0 + q : kc ? sid[q] : __ldcg(&glin[q]); };
        if (nr <= N) {                                // the last subcluster: all that is left
            if (t == 0) ctl->cnt_in[c] = n_live;
            if (!grid_sync(ctl, a.flags, gen)) return;
            uint32_t before = 0;
            for (uint32_t q = t; q < c; q += kThreads) before += __ldcg(&ctl->cnt_in[q]);
            before = block_sum(before);
            for (uint32_t q = t; q < n_live; q += kThreads) seg_out[before + q] = LID(q);
            break;
        }

        // ---- A: float32 distances of the points left and the first histogram
        for (int j = t; j < d; j += kThreads) Ls[j] = __uint_as_float(__ldcg(&ctl->Lbits[par][j]));
        const bool have_guess = guess != kGone;
        for (int b = t; b < (have_guess ? 2 : 1) * kHistBins; b += kThreads) dyn[b] = 0;
        if (c == 0 && t == 0) ctl->band_cnt[par ^ 1] = 0;
        if (Gl > 0 && c >= Gs && r > 0) {
            // the previous subcluster's points: marked removed, out of their buckets' counts
            // (this round's landmark needs both, its other CTAs have rows to read)
            const uint32_t *prev = a.perm + (r - 1) * a.N;
            for (uint32_t q = (c - Gs) * kThreads + t; q < N; q += (uint32_t)Gl * kThreads) {
                const uint32_t id = __ldcg(&prev[q]);
                a.key[id] = kGone;
                drop_buckets<D>(a.x, d, id, a.bcs, nbk);
            }
        }
        __syncthreads();
        // the key of one point of the round, stored for phases B-D and counted
        auto key_out = [&](bool live, uint32_t pos, uint32_t id, uint32_t k) {
            if (live) {
                a.key[id] = k;
                if (kc) skey[pos] = k;
                else a.kpos[s0 + pos] = k;
            }
            // the keys of a round crowd into a few bins: one shared atomic per bin and warp
            const uint32_t b = live ? (k >> 21) : kGone;
            const uint32_t peers = __match_any_sync(0xffffffffu, b);
            if (live && lane == __ffs(peers) - 1) atomicAdd(&sh[b], (uint32_t)__popc(peers));
            if (have_guess) {
                const uint32_t g2 = live && (k >> 21) == guess ? (k >> 10) & (kHistBins - 1) : kGone;
                const uint32_t pg = __match_any_sync(0xffffffffu, g2);
                if (g2 != kGone && lane == __ffs(pg) - 1) atomicAdd(&gh[g2], (uint32_t)__popc(pg));
            }
        };
        if constexpr (kCoopRows<D>()) {
            coop_keys<D>(a.x, Ls, n_live, s0, r == 0, kc, sid, glin, a.key, skey, a.kpos, sh, gh, guess);
        } else
        for (uint32_t base = 0; base < n_live; base += B * kThreads) {
            bool lv[B];
            uint32_t ids[B];
#pragma unroll
            for (int q = 0; q < B; q++) {
                const uint32_t qi = base + q * kThreads + t;
                lv[q] = qi < n_live;
                ids[q] = lv[q] ? LID(qi) : s0;
            }
            // past the end a thread reads the slice's first row again (an L1 hit), so every
            // thread keeps B rows in flight without branching
            float dl[B];
#pragma unroll
            for (int q = 0; q < B; q++) dl[q] = dist32<D>(a.x + (size_t)ids[q] * d, Ls, d);
#pragma unroll
            for (int q = 0; q < B; q++) key_out(lv[q], base + q * kThreads + t, ids[q], __float_as_uint(dl[q]));
        }
        __syncthreads();
        {
            uint32_t *hist0 = ctl->hist[par][0];
            for (int b = t; b < kHistBins; b += kThreads)
                if (sh[b]) atomicAdd(&hist0[b], sh[b]);
            if (have_guess) {
                uint32_t *gg = &ctl->ghist[par][0];
                for (int b = t; b < kHistBins; b += kThreads)
                    if (gh[b]) atomicAdd(&gg[b], gh[b]);
            }
        }
        if (!grid_sync(ctl, a.flags, gen)) return;

        // ---- B: the bin of the N-th key and the second digit inside it (the second
        // histogram is only built here when the bin was not guessed)
        uint32_t b0, rank0, b1 = 0, rank1 = 0;
        bool hit;
        find_bins(ctl->hist[par][0], have_guess ? ctl->ghist[par] : nullptr, guess, N - 1u, b0, rank0, b1,
                  rank1, hit);
        guess = b0;
        if (!hit) {
            uint32_t *hist1 = ctl->hist[par][1];
            for (int b = t; b < kHistBins; b += kThreads) sh[b] = 0;
            __syncthreads();
            for (uint32_t q0 = t; q0 < n_live; q0 += 4 * kThreads) {
                uint32_t k4[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t qi = q0 + q * kThreads;
                    k4[q] = qi >= n_live ? kGone : kc ? skey[qi] : __ldcg(&a.kpos[s0 + qi]);
                }
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if ((k4[q] >> 21) == b0 && k4[q] != kGone) atomicAdd(&sh[(k4[q] >> 10) & (kHistBins - 1)], 1u);
            }
            __syncthreads();
            for (int b = t; b < kHistBins; b += kThreads)
                if (sh[b]) atomicAdd(&hist1[b], sh[b]);
            if (!grid_sync(ctl, a.flags, gen)) return;
            find_bin(hist1, rank0, b1, rank1);
        }

        // ---- C: classify; the band is listed
        if (t == 0) band_cutoffs(b0, b1, d, s_in_key, s_out_key);
        {   // clear next round's histograms (last read in the previous round)
            uint32_t *nh = &ctl->hist[par ^ 1][0][0];
            for (uint32_t b = c * kThreads + t; b < 2u * kHistBins; b += G * kThreads) nh[b] = 0;
            uint32_t *ng = &ctl->ghist[par ^ 1][0];
            for (uint32_t b = c * kThreads + t; b < (uint32_t)kHistBins; b += G * kThreads) ng[b] = 0;
        }
        __syncthreads();
        const uint32_t in_key = s_in_key, out_key = s_out_key;
        auto to_band = [&](uint32_t qi, uint32_t k) {
            const uint32_t slot = atomicAdd(&ctl->band_cnt[par], 1u);
            a.band_k32[slot] = k;
            a.band_pos[slot] = LID(qi);
        };
        // keys from shared memory: 4 per thread at a time; from global memory: kCB
        uint32_t n_in = kc ? classify_keys<4>(n_live, in_key, out_key, [&](uint32_t qi) { return skey[qi]; }, to_band)
                           : classify_keys<kCB>(n_live, in_key, out_key,
                                                [&](uint32_t qi) { return __ldcg(&a.kpos[s0 + qi]); }, to_band);
        n_in = block_sum(n_in);
        if (t == 0) ctl->cnt_in[c] = n_in;
        if (!grid_sync(ctl, a.flags, gen)) return;

        // ---- D: settle the band, take the subcluster, next landmark
        // the per-CTA counts, the band's size and its first entries in one round trip
        const uint32_t nb = __ldcg(&ctl->band_cnt[par]);
        uint32_t sk[kBandStage / kThreads], sp[kBandStage / kThreads];
#pragma unroll
        for (int r = 0; r < kBandStage / kThreads; r++) {
            const uint32_t q = t + r * kThreads;
            sk[r] = q < n ? __ldcg(&a.band_k32[q]) : 0u;
            sp[r] = q < n ? __ldcg(&a.band_pos[q]) : 0u;
        }
        uint32_t all_in, in_before;
        {
            uint32_t va = 0, vb = 0, e0, e1;
            for (uint32_t q = t; q < G; q += kThreads) {
                const uint32_t v = __ldcg(&ctl->cnt_in[q]);
                va += v;
                if (q < c) vb += v;
            }
            block_excl_scan2(va, vb, e0, e1, all_in, in_before);
        }
        const bool staged = nb <= (uint32_t)kBandStage;
        if (staged) {
#pragma unroll
            for (int r = 0; r < kBandStage / kThreads; r++) {
                const uint32_t q = t + r * kThreads;
                if (q < nb) {
                    s_bk[q] = sk[r];
                    s_bp[q] = sp[r];
                }
            }
            __syncthreads();
        }
        auto BK = [&](uint32_t q) { return staged ? s_bk[q] : __ldcg(&a.band_k32[q]); };
        auto BP = [&](uint32_t q) { return staged ? s_bp[q] : __ldcg(&a.band_pos[q]); };
        const uint32_t need = N > all_in ? N - all_in : 0u;
        if ((all_in > N || need > nb) && c == 0 && t == 0) atomicOr(&a.flags[1], 1u);
        uint32_t lo = in_key, tout = 0, ntt = 0;       // the rule (see taken())
        uint32_t band_before = 0;
        bool slow = false;
        if (need > 0 && need < nb) {
            // Fast path, in shared memory (every CTA redundantly).  The need-th smallest
            // float32 key T32 of the band comes from a one-ulp histogram; the float32 error
            // bound around T32 leaves a tight set of a few entries; their distances in
            // compensated float32 (dff, within eps_ff of the float64 definition) settle all
            // of them but those within the dff error of the cut-off (in practice only exact
            // ties), which are decided in float64.
            const uint32_t range = out_key - in_key + 1u;
            // the tight set spans about 2(d+4) of the band's `range` one-ulp keys: when the
            // band is dense enough that it would hold over twice kTight entries, the fast
            // path cannot succeed and is skipped (a choice of path, not of result)
            slow = range > (uint32_t)kBandBins ||
                   (uint64_t)nb * (uint64_t)(2 * (d + 4)) > (uint64_t)(2 * kTight) * range;
            if (!slow) {
                for (int b = t; b < kBandBins; b += kThreads) hb[b] = 0;
                if (t == 0) {
                    s_nt = 0;
                    s_na = 0;
                }
                __syncthreads();
                for (uint32_t q = t; q < nb; q += kThreads) atomicAdd(&hb[BK(q) - in_key], 1u);
                __syncthreads();
                {   // the one-ulp bin of the need-th smallest band key
                    constexpr int per = kBandBins / kThreads;
                    uint32_t loc = 0;
#pragma unroll
                    for (int q = 0; q < per; q++) loc += hb[t * per + q];
                    uint32_t tot;
                    const uint32_t before = block_excl_scan(loc, tot);
                    const uint32_t target = need - 1;
                    if (target >= before && target < before + loc) {
                        uint32_t cc = before;
                        for (int q = 0; q < per; q++) {
                            const uint32_t h = hb[t * per + q];
                            if (target >= cc && target < cc + h) s_t32 = in_key + (uint32_t)(t * per + q);
                            cc += h;
                        }
                    }
                }
                __syncthreads();
                uint32_t tin, tt;
                band_cutoffs_key(s_t32, s_t32, d, tin, tt);
                uint32_t n_cert = 0, cert_before = 0;
                for (uint32_t q = t; q < nb; q += kThreads) {
                    const uint32_t k = BK(q);
                    const uint32_t pq = BP(q);
                    if (k < tin) {
                        n_cert++;
                        cert_before += pq < s0;
                    } else if (k <= tt) {
                        const uint32_t slot = atomicAdd(&s_nt, 1u);
                        if (slot < (uint32_t)kTight) tpos[slot] = pq;
                    }
                }
                n_cert = block_sum(n_cert);
                const uint32_t nt = s_nt;
                slow = nt > (uint32_t)kTight || n_cert > need || need - n_cert > nt;
                if (!slow) {
                    const uint32_t need2 = need - n_cert;
                    for (uint32_t q = t; q < nt; q += kThreads) {
                        float h, l;
                        dist_ff(a.x + (size_t)tpos[q] * d, Ls, d, h, l);
                        th[q] = h;
                        tl[q] = l;
                    }
                    __syncthreads();
                    // V: the tight entry of rank need2-1 in (dff, index) order
                    for (uint32_t q = t; q < nt; q += kThreads) {
                        uint32_t rk = 0;
                        for (uint32_t o = 0; o < nt; o++)
                            rk += (uint32_t)((th[o] < th[q]) |
                                             ((th[o] == th[q]) & ((tl[o] < tl[q]) | ((tl[o] == tl[q]) & (tpos[o] < tpos[q])))));
                        if (rk == need2 - 1) s_v = q;
                    }
                    __syncthreads();
                    // the need2-th smallest delta64 lies within eps*hv of hv (order statistics
                    // move by at most the per-entry error); an entry is decided if its own
                    // error cannot bridge the gap (plus an absolute floor against underflow)
                    const float hv = th[s_v], lv = tl[s_v];
                    const float win = 2.0f * eps_ff(d) * hv + 0x1p-120f;
                    uint32_t n_take = 0;
                    for (uint32_t q = t; q < nt; q += kThreads) {
                        const float diff = __fadd_rn(__fsub_rn(th[q], hv), __fsub_rn(tl[q], lv));
                        const uint32_t cls = diff < -win ? 1u : 0u;
                        if (diff >= -win && diff <= win) {
                            const uint32_t slot = atomicAdd(&s_na, 1u);
                            tamb[slot] = q;
                        }
                        n_take += cls;
                        tcls[q] = cls;
                    }
                    n_take = block_sum(n_take);
                    const uint32_t na = s_na;
                    const uint32_t need3 = need2 >= n_take ? need2 - n_take : 0u;
                    if (need3 > na && t == 0) atomicOr(&a.flags[1], 1u);
                    if (need3 >= na) {
                        for (uint32_t q = t; q < na; q += kThreads) tcls[tamb[q]] = 1u;
                    } else if (need3 > 0) {
                        for (uint32_t q = t; q < na; q += kThreads)
                            td[q] = (unsigned long long)__double_as_longlong(dist64(a.x + (size_t)tpos[tamb[q]] * d, Ls, d));
                        __syncthreads();
                        for (uint32_t q = t; q < na; q += kThreads) {
                            const unsigned long long kq = td[q];
                            const uint32_t pq = tpos[tamb[q]];
                            uint32_t rk = 0;
                            for (uint32_t o = 0; o < na; o++) rk += (td[o] < kq) || (td[o] == kq && tpos[tamb[o]] < pq);
                            tcls[tamb[q]] = rk < need3 ? 1u : 0u;
                        }
                    }
                    lo = max(in_key, tin);
                    tout = tt;
                    ntt = nt;
                }
                __syncthreads();
                if (!slow) {                       // taken band points before the slice
                    band_before = cert_before;
                    for (uint32_t q = t; q < nt; q += kThreads) band_before += tcls[q] != 0 && tpos[q] < s0;
                }
            }
            if (slow) {
                // wide band (e.g. many equal distances): float64 for every band entry, spread
                // evenly over all CTAs (entry q on CTA q mod G: the float64 pipe is the
                // bound), then one CTA selects while the rest wait
                for (uint32_t q = t * G + c; q < nb; q += G * kThreads) {
                    const uint32_t pq = __ldcg(&a.band_pos[q]);
                    a.band_key[q] = (uint64_t)__double_as_longlong(dist64(a.x + (size_t)pq * d, Ls, d));
                }
                if (!grid_sync(ctl, a.flags, gen)) return;
                uint64_t K = 0;
                uint32_t Pp = 0;
                if (c == 0) {
                    // the band's float64 keys, the fast path's arrays and the key cache are
                    // no longer needed here: the selection may use that shared memory
                    if (!select_band_fast(a.band_key, a.band_pos, nb, need, dyn, K, Pp))
                        select_band_global(a.band_key, a.band_pos, nb, need, K, Pp);
                    if (t == 0) {
                        ctl->sel_key = K;
                        ctl->sel_pos = Pp;
                    }
                }
                if (!grid_sync(ctl, a.flags, gen)) return;
                K = __ldcg(&ctl->sel_key);
                Pp = __ldcg(&ctl->sel_pos);
                for (uint32_t q0 = t; q0 < nb; q0 += kSelBatch * kThreads) {
                    uint64_t kq[kSelBatch];
                    uint32_t pq[kSelBatch];
#pragma unroll
                    for (int u = 0; u < kSelBatch; u++) {
                        const uint32_t q = q0 + u * kThreads;
                        kq[u] = q < nb ? __ldcg(&a.band_key[q]) : ~0ull;
                        pq[u] = q < nb ? __ldcg(&a.band_pos[q]) : n;
                    }
#pragma unroll
                    for (int u = 0; u < kSelBatch; u++) {
                        if (kq[u] < K || (kq[u] == K && pq[u] <= Pp)) {
                            if (pq[u] < s0) band_before++;
                            else if (pq[u] < s1) a.key[pq[u]] = kTaken;
                        }
                    }
                }
                lo = in_key;
                tout = 0;
                ntt = 0;
            }
        } else if (need > 0) {
            lo = out_key + 1u;      // need >= nb: the whole band is taken (need > nb is flagged)
            for (uint32_t q = t; q < nb; q += kThreads) band_before += BP(q) < s0;
        }
        const Rule R{lo, tout, ntt, tpos, tcls};
        band_before = block_sum(band_before);       // its barriers also publish the kTaken marks
        // take the subcluster: ids in ascending order to the segment, the rest stay listed;
        // a taken point is marked removed and leaves the live count of its d buckets
        // (with landmark-only CTAs they do that bookkeeping in the next round's phase A)
        n_live -= compact_list(LID, n_live, seg_out + in_before + band_before, kc ? sid : a.lidx + (size_t)(par ^ 1) * n + s0,
                               [&](uint32_t qi, uint32_t id) {
                                   uint32_t k = kc ? skey[qi] : __ldcg(&a.kpos[s0 + qi]);
                                   // a wide band marks its taken points in key[] by id: only a
                                   // key inside the band needs that look-up
                                   if (slow && k >= in_key && k <= out_key) k = __ldcg(&a.key[id]);
                                   return taken(R, k, id);
                               },
                               [&](uint32_t id) {
                                   if (Gl == 0) {
                                       a.key[id] = kGone;
                                       drop_buckets<D>(a.x, d, id, a.bcs, nbk);
                                   }
                               });

        // next landmark.  Bucket live counts are upper bounds (this round's removals are
        // not counted yet), and a point counts as left only if it is neither marked removed
        // nor taken by this round's rule (a key read before or after its owner marks it
        // gives the same answer).  After a wide band its kTaken marks are published first.
        if (slow && !grid_sync(ctl, a.flags, gen)) return;
        const Rule &RL = R;
        for (int j = lm_first; j >= 0 && j < d; j += lm_step) {
            const uint4 *bj = a.bcs + (size_t)j * nbk;
            const uint32_t *oj = a.ord + (size_t)j * a.ord_ld;
            uint32_t b = __ldcg(&ctl->lptr[j]);       // the buckets before b hold no point left
            uint32_t mnb = kGone;
            while (b < nbk) {
                // the first bucket from b on with a live count
                const uint32_t bb = b + (uint32_t)t;
                const uint4 e = bb < nbk ? __ldcg(&bj[bb]) : make_uint4(0u, 0u, 0u, 0u);
                uint32_t fb = warp_min(e.x > 0 ? bb : kGone);
                if (lane == 0) red_a[w] = fb;
                __syncthreads();
                fb = red_a[0];
#pragma unroll
                for (int q = 1; q < W; q++) fb = min(fb, red_a[q]);
                if (bb == fb) {
                    s_st = e.y;
                    s_en = e.z;
                }
                __syncthreads();
                if (fb == kGone) {
                    b += kThreads;
                    continue;
                }
                // the smallest value among its entries left
                const uint32_t st = s_st, en = s_en;
                uint32_t lm = kGone;
                for (uint32_t q = st + t; q < en; q += kThreads) {
                    const uint32_t id = __ldcg(&oj[q]);
                    const uint32_t k = __ldcg(&a.key[id]);
                    const uint32_t xv = __float_as_uint(__ldg(&a.x[(size_t)id * d + j]));
                    if (k != kGone && !taken(RL, k, id)) lm = min(lm, xv);
                }
                lm = warp_min(lm);
                if (lane == 0) red_b[w] = lm;
                __syncthreads();
                lm = red_b[0];
#pragma unroll
                for (int q = 1; q < W; q++) lm = min(lm, red_b[q]);
                __syncthreads();
                if (lm != kGone) {
                    mnb = lm;
                    b = fb;
                    break;
                }
                b = fb + 1;                            // every entry of fb is gone
            }
            if (t == 0) {
                ctl->lptr[j] = b;
                ctl->Lbits[par ^ 1][j] = mnb == kGone ? kInfBits : mnb;
            }
        }
        if (!grid_sync(ctl, a.flags, gen)) return;
    }
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
cudaError_t peel_launch(const PeelBuffers &b, int64_t n, int d, int64_t N, int sm_count,
                        cudaStream_t st, KTimer *kt)
{
    const int64_t S = (n + N - 1) / N;
    // all control state starts cleared; round 0's landmark is the origin (the scaled
    // minimum of every attribute is exactly 0)
    cudaError_t e = cudaMemsetAsync(b.ctl, 0, sizeof(PeelCtl), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b.bcnt, 0, (size_t)d * b.nbuckets * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const size_t smem = kPeelDynWords * sizeof(uint32_t);
    e = cudaFuncSetAttribute(k_peel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel<D>, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)sm_count * std::min(per_sm, 4);
    if (grid > kMaxPeelGrid) grid = kMaxPeelGrid;
    const int64_t want = (n + 63) / 64;             // at least ~64 points per CTA
    if (grid > want) grid = std::max<int64_t>(1, want);
    PeelArgs a;
    a.x = b.x;
    a.d = d;
    a.n = n;
    a.N = N;
    a.S = S;
    a.key = b.key;
    a.ord = b.ord;
    a.bcnt = b.bcnt;
    a.bcs = b.bcs;
    a.lidx = b.lidx;
    a.kpos = b.kpos;
    a.ord_ld = b.ord_ld;
    a.nbk = b.nbuckets;
    a.band_key = b.band_key;
    a.band_k32 = b.band_k32;
    a.band_pos = b.band_pos;
    a.perm = b.perm;
    a.landmarks = b.landmarks;
    a.ctl = b.ctl;
    a.flags = b.flags;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    kt->begin(st);
    e = cudaLaunchKernelEx(&cfg, k_peel<D>, a);
    kt->end(PSCL_K_PEEL, st);
    if (e != cudaSuccess) return e;
    return launch_gather(b.x, b.perm, n, d, b.xseg, sm_count, st, kt);
}

}  // namespace

cudaError_t launch_gather(const float *x, const uint32_t *perm, int64_t n, int d, float *xseg, int sm_count,
                          cudaStream_t st, KTimer *kt)
{
    int64_t work = (d % 4 == 0) ? n * d / 4 : n * d;
    int64_t g = (work + 255) / 256;
    if (g > (int64_t)sm_count * 16) g = (int64_t)sm_count * 16;
    if (g < 1) g = 1;
    kt->begin(st);
    if (d % 4 == 0)
        k_gather_rows<true><<<(int)g, 256, 0, st>>>(x, perm, n, d, xseg);
    else
        k_gather_rows<false><<<(int)g, 256, 0, st>>>(x, perm, n, d, xseg);
    kt->end(PSCL_K_GATHER, st);
    return cudaGetLastError();
}

uint32_t peel_buckets(int64_t n)
{
    uint32_t nb = 4096;
    while (nb < 65536u && (int64_t)nb * 16 < n) nb <<= 1;
    return nb;
}

cudaError_t launch_peel(const PeelBuffers &b, int64_t n, int d, int64_t N, int sm_count,
                        cudaStream_t st, KTimer *kt)
{
    switch (d) {
    case 2: return peel_launch<2>(b, n, d, N, sm_count, st, kt);
    case 4: return peel_launch<4>(b, n, d, N, sm_count, st, kt);
    case 8: return peel_launch<8>(b, n, d, N, sm_count, st, kt);
    case 16: return peel_launch<16>(b, n, d, N, sm_count, st, kt);
    case 32: return peel_launch<32>(b, n, d, N, sm_count, st, kt);
    case 64: return peel_launch<64>(b, n, d, N, sm_count, st, kt);
    case 128: return peel_launch<128>(b, n, d, N, sm_count, st, kt);
    default: return peel_launch<0>(b, n, d, N, sm_count, st, kt);
    }
}

}  // namespace pscl
