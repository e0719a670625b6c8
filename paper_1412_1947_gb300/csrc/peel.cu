// Equal-sized subclustering (Algorithm 1 steps 2-5, repeated on the points left out as
// §II describes): round r builds the landmark L = per-attribute minimum of the
// remaining points, takes the N remaining points nearest to L as subcluster r and
// removes them.
//
// Membership is defined by the float64 distance
//     delta64_i = sum_{j ascending} (double(x_ij) - double(L_j))^2   (one rounding per op)
// with equal distances taken in ascending point index.
//
// Epochs.  L changes only when every remaining point that holds some attribute's minimum
// has been taken, and while L stays the distances stay: the round after r takes the next N
// points of the same order.  So one pass of distances serves an epoch of up to K rounds
// (K = rounds_per_pass, at most kMaxEpoch): with K boundaries at ranks N, 2N, ..., KN of
// the order by (delta64, index), every point left gets the round of the epoch it falls
// in, and the epoch commits its rounds up to the first one after which some attribute
// has no holder of its landmark value left.  The later rounds' assignments are dropped
// and the next epoch starts from the new landmark (a new pass of distances) or, when all
// K rounds committed, from the same one (no pass at all).  K itself is read off the keys:
// the holders' largest key per attribute bounds the round in which the landmark changes,
// so an epoch resolves only the boundaries up to there (see resolve_cutoffs).  On the
// headline workload (2^20 points, 16 attributes, 256 rounds) the landmark changes in 50
// rounds, and the peel runs 50 epochs.
//
// Each pass works in float32 and keeps exact arithmetic for thin bands around the
// boundaries:
//   A. delta32_i in float32 (FMA chains, a row's pieces summed across the lanes that read
//      it), kept as its bit pattern (order-preserving for non-negative floats), and a
//      2048-bin histogram of key bits 31..21.  Points equal to L in an attribute are
//      counted per attribute and flagged (the holders);
//   B. per boundary, the first-digit bin holding its rank, and 2048-bin histograms of
//      bits 20..10 inside those bins: each boundary's float32 key lies in a 22-bit prefix
//      [A, B];
//   C. |delta32 - delta64| <= eps*delta32 + ea with eps = (d+4)*2^-23, ea = 2^-120, so the
//      boundary's delta64 lies in [A(1-eps)-ea, B(1+eps)+ea]: a point whose bound lies
//      below that interval is certainly before the boundary, one above it certainly
//      after; the few in between form the boundary's band (boundaries whose bands overlap
//      form one group);
//   D. each group is settled by one CTA: compensated float32 distances of its entries
//      (within eps_ff of delta64) order all but the entries within that error of a cut,
//      and those (in practice exact ties) are ranked by float64 and index.
// The partition is therefore exactly the float64 definition's, whatever float32 does.
//
// Most landmark changes move one or two attributes (the others keep a holder).  The pass
// after such a change reads only the attributes that moved: with J those attributes, o_j
// the old and l_j the new value, the squared distance changes by exactly
//     sum_{j in J} (l_j - o_j)(l_j + o_j - 2 x_j),
// which is added to every live key in float32.  The keys' error bound then takes the form
// |delta32 - delta64| <= eps*delta32 + ea with eps and ea carried from pass to pass: a
// full pass sets (eps0, ea0) = ((d+4) 2^-23, 2^-120), and an update with C = sum_J (l_j - o_j)
// gives eps' = eps + 2^-23 and ea' = ea + (5 eps + (16 + 4|J|) 2^-24) C (the update's own
// rounding, the old key's error carried to the new key, and the float64 definition's;
// scaled values lie in [0, 1]).  Phase C uses the carried bound; a full pass is taken
// instead when J spans many 32-byte sectors of a row, when more than kIncMax attributes
// moved, or when eps would pass 1.5 eps0 or ea an eighth of eps0 times the last epoch's
// first boundary key (the landmark sits at the corner of the minima, so the boundary keys
// are large and ea stays a small share of the bands' width).
//
// Points never move: CTA c owns the index slice [c n/G, (c+1) n/G) and keeps the ids of its
// points left in a list, in ascending order, with their keys by list position.  Every
// point gets its round in rnd[]; after the launch a stable counting sort by round packs
// the subclusters (ascending index inside each).  The next landmark needs no pass over
// the rows: before the first epoch a counting sort lists, per attribute, the point ids by
// value bucket (buckets are monotone in the value); the minimum over the points left is
// the smallest value left in the first bucket that still has a point left, and one bucket
// pointer per attribute only moves forward (the buckets it passes hold no point left, and
// points never come back), so each bucket emptied by removals is read once more in all.
//
// All epochs run in one persistent cooperative launch, the phases separated by grid
// barriers.  Every barrier wait is bounded; a CTA that gives up sets the abort flag, every
// other CTA then leaves at its next wait, and the host sees PSCL_ETIMEOUT.
#include <algorithm>

#include "pscl_internal.cuh"

namespace pscl {
namespace {

constexpr int kThreads = 256;
constexpr int kW = kThreads / 32;
constexpr uint32_t kInfBits = 0x7f800000u;
constexpr uint32_t kGone = 0xFFFFFFFFu;       // key past the end of a list
constexpr uint32_t kNone = 0xFFFFFFFFu;       // round of a point not assigned (yet)
constexpr int kBkGroup = 16;                   // attributes per sweep of the bucket build
constexpr int kBkUnroll = 4;                   // (point, attribute) pairs per thread at a time
constexpr int kIncMax = 8;                     // moved attributes a pass may update keys for
constexpr int kKeyCache = 4096;               // keys and ids of a slice kept in shared memory, if it fits
constexpr int kSelBins = 2048;
constexpr int kSelList = 1024;
constexpr int kSelBatch = 8;
constexpr int kStage = 1024;                  // band entries of one group staged in shared memory
constexpr int kStageOff = kSelBins + 3 * kSelList;
constexpr int kScrWords = kStageOff + 3 * kStage;
static_assert(kScrWords >= kHistBins, "phase A's histogram fits the scratch");
static_assert(kStageOff % 2 == 0, "staged 64-bit keys are 8-byte aligned");
constexpr int kPeelDynWords = kScrWords + 2 * kKeyCache + kKeyCache / 4;
constexpr int kQT = 8;                        // tiles of kThreads items per compaction scan
constexpr int kCB = 8;                        // keys per thread in flight when classifying
constexpr int kHoldBatch = 8;                 // state bytes per thread in flight when finding holders
// State byte of each list position: bit 7 set once the point has held some attribute's
// landmark value (it then holds it while it is left); bits 0..6 its place in the current
// epoch: a round 0..kMaxEpoch-1 it is certainly in, kFlBand (in a band), kFlNone.
constexpr uint8_t kFlHold = 0x80;
constexpr uint8_t kFlBand = 0x7E;
constexpr uint8_t kFlNone = 0x7F;
constexpr uint32_t kPosMask = 0x7FFFFFFFu;    // a band entry's id; bit 31 carries its hold flag
constexpr int kDefaultRounds = 32;            // rounds per distance pass by default
constexpr int kSlotsSmem = kScrWords / kHistBins;   // second-digit histograms counted in shared memory
constexpr unsigned kDefaultSpin = 1u << 25;   // ~1-2 s of polling per barrier at most

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
    __shared__ uint32_t wsum[kW];
    __shared__ uint32_t wtot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < kW ? wsum[lane] : 0;
        uint32_t si = warp_incl_scan(s);
        if (lane < kW) wsum[lane] = si - s;
        if (lane == kW - 1) wtot = si;
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

__device__ __forceinline__ uint32_t warp_min(uint32_t v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ uint32_t block_min(uint32_t v)
{
    __shared__ uint32_t wm[kW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_min(v);
    if (lane == 0) wm[w] = v;
    __syncthreads();
    v = wm[0];
#pragma unroll
    for (int q = 1; q < kW; q++) v = min(v, wm[q]);
    __syncthreads();
    return v;
}

// ------------------------------------------------------------------ grid barriers
// Thread 0's bounded wait for the arrival counter to reach `target`.  Returns false if the
// launch is being aborted (or this wait gave up, which aborts it).
__device__ bool bar_wait(PeelCtl *ctl, uint32_t *flags, unsigned target, unsigned limit)
{
    unsigned spins = 0, v;
    for (;;) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&ctl->bar_count) : "memory");
        if ((int)(v - target) >= 0) return true;
        if ((++spins & 63) == 0) {
            if (*(volatile unsigned *)&ctl->abort) return false;
            if (spins > limit) {
                atomicExch(&ctl->abort, 1u);
                atomicOr(&flags[1], 2u);               // timed out
                return false;
            }
            __nanosleep(32);
        }
    }
}

// Grid-wide barrier with a bounded wait: a monotonic arrival counter (release on arrival,
// acquire while polling), so no reset is needed within a launch.  `extra` arrivals more
// than the grid gives are awaited (a test of the give-up path; 0 otherwise).
__device__ bool grid_sync(PeelCtl *ctl, uint32_t *flags, unsigned &target, unsigned limit, unsigned extra = 0)
{
    __shared__ int ok;
    target += gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blockIdx.x == 0) ctl->barriers += 1;     // statistics (one writer)
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar_count) : "memory");
        ok = bar_wait(ctl, flags, target + extra, limit) ? 1 : 0;
    }
    __syncthreads();
    return ok != 0;
}

// A grid barrier whose last arriving CTA runs work() (all its threads) before any CTA
// leaves: every CTA adds one arrival, the last one then runs the work and adds one more.
template <class Work>
__device__ bool grid_sync_last(PeelCtl *ctl, uint32_t *flags, unsigned &target, unsigned limit, Work work)
{
    __shared__ int ok, last;
    target += gridDim.x + 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blockIdx.x == 0) ctl->barriers += 1;     // statistics (one writer)
        unsigned old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(&ctl->bar_count) : "memory");
        last = old == target - 2u;
    }
    __syncthreads();
    if (last) {
        work();
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar_count) : "memory");
            ok = *(volatile unsigned *)&ctl->abort ? 0 : 1;
        }
    } else if (threadIdx.x == 0) {
        ok = bar_wait(ctl, flags, target, limit) ? 1 : 0;
    }
    __syncthreads();
    return ok != 0;
}

// ------------------------------------------------------------------ distances
// float32 distance of one row by one thread (the phase-A path for d not a multiple of 4,
// or below 8): t = RN(x - L), acc = RN(t*t + acc) (fused), ascending attributes.  `hz` is
// set when some attribute equals the landmark's.
template <int D>
__device__ __forceinline__ float dist32(const float *__restrict__ row, const float *Ls, int d, bool &hz)
{
    float acc = 0.0f;
    bool z = false;
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
            z |= (t0 == 0.0f) | (t1 == 0.0f) | (t2 == 0.0f) | (t3 == 0.0f);
        }
    } else {
        const int dd = D > 0 ? D : d;
#pragma unroll 4
        for (int j = 0; j < dd; j++) {
            float t = __fsub_rn(__ldg(&row[j]), Ls[j]);
            acc = __fmaf_rn(t, t, acc);
            z |= t == 0.0f;
        }
    }
    hz = z;
    return acc;
}

// float64 distance exactly as defined: diff, square, add, each rounded, no fusion.
__device__ double dist64(const float *__restrict__ row, const float *Ls, int d)
{
    double s = 0.0;
    for (int j = 0; j < d; j++) {
        double diff = __dsub_rn((double)__ldg(&row[j]), (double)Ls[j]);
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
#pragma unroll 4
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

// The compensated distance h + l rounded once to float64 (its bit pattern orders like
// the value), the key a group's entries are ranked by.
__device__ __forceinline__ uint64_t dff_key(const float *__restrict__ row, const float *Ls, int d)
{
    float h, l;
    dist_ff(row, Ls, d, h, l);
    double v = __dadd_rn((double)h, (double)l);
    if (!(v > 0.0)) v = 0.0;
    return (uint64_t)__double_as_longlong(v);
}

// Cut-offs of phase C from the 22-bit key prefix [A, B] of a boundary's float32 key.
// With |delta32 - delta64| <= eps delta32 + ea (eps <= 1/3) the boundary's delta64 lies in
// [A(1-eps) - ea, B(1+eps) + ea]; a point is certainly before it if delta32 (1+eps) + ea
// is below that interval, which holds for delta32 < A(1-2eps) - 2ea, and certainly after
// it if delta32 (1-eps) - ea is above it, which holds for delta32 > B(1+3eps) + 3ea.  Both
// cut-offs are evaluated in float32 rounded towards the safe side.
__device__ void band_cutoffs(uint32_t b0, uint32_t b1, float eps, float ea, uint32_t &in_key, uint32_t &out_key)
{
    const uint32_t lo = (b0 << 21) | (b1 << 10), hi = lo | 0x3FFu;
    const float A = __uint_as_float(lo), B = __uint_as_float(hi);
    const float in_thr = __fsub_rd(__fmul_rd(A, __fsub_rd(1.0f, 2.0f * eps)), 2.0f * ea);
    const float out_thr = __fadd_ru(__fmul_ru(B, __fadd_ru(1.0f, __fmul_ru(3.0f, eps))), __fmul_ru(3.0f, ea));
    in_key = in_thr > 0.0f ? __float_as_uint(in_thr) : 0u;
    out_key = __float_as_uint(out_thr);
}

// ------------------------------------------------------------------ exact selection
// The `need`-th smallest (1-based) of nb entries by (key, position), key_at / pos_at giving
// entry i.  Single-block radix select with 8-bit digits over the 96-bit composite.
template <class KeyAt, class PosAt>
__device__ void select_radix(KeyAt key_at, PosAt pos_at, uint32_t nb, uint32_t need, uint64_t &K, uint32_t &Pp)
{
    __shared__ uint32_t h[256];
    __shared__ uint64_t pk;
    __shared__ uint32_t pp, rank;
    if (threadIdx.x == 0) {
        pk = 0;
        pp = 0;
        rank = need - 1;
    }
    __syncthreads();
    for (int pass = 0; pass < 12; pass++) {
        h[threadIdx.x] = 0;
        __syncthreads();
        const uint64_t cpk = pk;
        const uint32_t cpp = pp;
        for (uint32_t i = threadIdx.x; i < nb; i += kThreads) {
            const uint64_t k = key_at(i);
            const uint32_t p = pos_at(i);
            bool match;
            uint32_t digit;
            if (pass < 8) {
                match = pass == 0 || (k >> (64 - 8 * pass)) == (cpk >> (64 - 8 * pass));
                digit = (uint32_t)(k >> (56 - 8 * pass)) & 0xFFu;
            } else {
                const int q = pass - 8;
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

// The same selection in three passes when the keys spread: the smallest and largest key
// give the bits all keys share; an 11-bit histogram of the next bits finds the digit of
// the need-th entry; that digit's entries (at most kSelList) are gathered in shared memory
// and ranked there by (key, position).  Returns false, with nothing decided, when all keys
// are equal or the digit holds more entries: the caller then runs select_radix.
// scratch: kSelBins + 3 kSelList words of shared memory.
template <class KeyAt, class PosAt>
__device__ bool select_fast(KeyAt key_at, PosAt pos_at, uint32_t nb, uint32_t need, uint32_t *scratch, uint64_t &K,
                            uint32_t &Pp)
{
    __shared__ unsigned long long s_mn[kW], s_mx[kW];
    __shared__ uint32_t s_bin, s_rank, s_cnt, s_hit;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t *h = scratch;
    uint64_t *lk = reinterpret_cast<uint64_t *>(scratch + kSelBins);      // 8-byte aligned: kSelBins is even
    uint32_t *lp = scratch + kSelBins + 2 * kSelList;
    unsigned long long mn = ~0ull, mx = 0ull;
    for (uint32_t i0 = t; i0 < nb; i0 += kSelBatch * kThreads) {
        unsigned long long kk[kSelBatch];
#pragma unroll
        for (int u = 0; u < kSelBatch; u++) {
            const uint32_t i = i0 + u * kThreads;
            kk[u] = i < nb ? key_at(i) : 0ull;
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
    for (int q = 1; q < kW; q++) {
        mn = min(mn, (unsigned long long)s_mn[q]);
        mx = max(mx, (unsigned long long)s_mx[q]);
    }
    __syncthreads();
    if (mn == mx) return false;                          // uniform across the block
    const int hb = 63 - __clzll((long long)(mn ^ mx));   // highest bit where keys differ
    const int sh = hb >= 10 ? hb - 10 : 0;               // digit = bits [sh, hb]
    for (uint32_t i0 = t; i0 < nb; i0 += kSelBatch * kThreads) {
        unsigned long long kk[kSelBatch];
#pragma unroll
        for (int u = 0; u < kSelBatch; u++) {
            const uint32_t i = i0 + u * kThreads;
            kk[u] = i < nb ? key_at(i) : 0ull;
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
    for (uint32_t i0 = t; i0 < nb; i0 += kSelBatch * kThreads) {
        unsigned long long kk[kSelBatch];
#pragma unroll
        for (int u = 0; u < kSelBatch; u++) {
            const uint32_t i = i0 + u * kThreads;
            kk[u] = i < nb ? key_at(i) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kSelBatch; u++) {
            const uint32_t i = i0 + u * kThreads;
            if (i < nb && ((uint32_t)(kk[u] >> sh) & (kSelBins - 1)) == bin) {
                const uint32_t slot = atomicAdd(&s_hit, 1u);
                lk[slot] = kk[u];
                lp[slot] = pos_at(i);
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

template <class KeyAt, class PosAt>
__device__ void select_kth(KeyAt key_at, PosAt pos_at, uint32_t nb, uint32_t need, uint32_t *scratch, uint64_t &K,
                           uint32_t &Pp)
{
    if (!select_fast(key_at, pos_at, nb, need, scratch, K, Pp)) select_radix(key_at, pos_at, nb, need, K, Pp);
}

// ------------------------------------------------------------------ buckets
// Bucket of a scaled value (in [0, 1]) among nb equal buckets: monotone in the value.
__device__ __forceinline__ uint32_t bucket_of(float v, uint32_t nb)
{
    v = fminf(fmaxf(v, 0.0f), 1.0f);
    const uint32_t b = __float2uint_rz(v * (float)nb);
    return b < nb ? b : nb - 1u;
}

// ------------------------------------------------------------------ the kernel
struct PeelArgs {
    const float *x;
    const float *xt;             // d x n: the points by attribute (or NULL: the updates read x)
    int d;
    int64_t n, N, S;
    uint32_t *rnd;
    uint8_t *pflag;              // 2 x n: the state byte of each list position
    uint32_t *ord;               // d x ord_ld: point ids by value bucket, per attribute
    uint32_t *bcnt;              // d x nbk: bucket counts, then cursors (zeroed before)
    uint4 *bcs;                  // d x nbk: (points left, first entry, end entry, 0)
    uint32_t *lidx;              // 2 x n: per CTA slice, the ids of its points left (not kc; two lists)
    uint32_t *kpos;              // 2 x n: their keys by list position
    int64_t ord_ld;
    uint32_t nbk;
    uint32_t *band_k32;
    uint32_t *band_pos;
    uint64_t *gkey;
    uint32_t *gpos;
    uint64_t *akey;
    uint32_t *apos;
    float *landmarks;            // S x d or NULL
    PeelCtl *ctl;
    uint32_t *flags;             // job flags: [1] |= 1 bound violated, 2 barrier timed out
    uint32_t kmax;               // rounds per distance pass
    uint32_t spin;               // polls of a barrier wait before it gives up
    uint32_t stall;              // test hook: the first barrier awaits one arrival too many
};

// rows a thread keeps in flight at once (64 floats of rows at most)
template <int D>
__host__ __device__ constexpr int kPeelBatch()
{
    return D <= 0 ? 1 : (D >= 64 ? 1 : (64 / D > 4 ? 4 : 64 / D));
}

// Phase A reads a row with P = min(D/4, 32) lanes, one float4 each (F per lane when D > 128),
// so that one warp load covers 32/P whole rows instead of one 16-byte piece of 32 rows.
// Each lane sums its part of P rows (fused, ascending attributes) and a butterfly over the
// P lanes leaves every lane the whole sum of one row.  Every squared difference passes
// through at most D/P + log2 P roundings, fewer than the d of the recursive sum that the
// phase-C error bound allows.
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

__device__ __forceinline__ bool in_mask(const uint32_t *jm, int j)
{
    return (jm[j >> 5] >> (j & 31)) & 1u;
}

// A live point equal to the landmark in some attribute: counted per such attribute whose
// landmark value is new (jm; the counts of the others carry over) and flagged for the
// epochs' holder bookkeeping.
__device__ __forceinline__ void note_holder(const float *__restrict__ row, const float *Ls, int d, uint8_t *fl,
                                            uint32_t *chold, const uint32_t *jm)
{
    for (int j = 0; j < d; j++)
        if (__ldg(&row[j]) == Ls[j] && in_mask(jm, j)) atomicAdd(&chold[j], 1u);
    *fl |= kFlHold;
}

// Phase A: every live point's float32 key, stored by list position (shared memory when
// kc, else kpos: the slice's keys) and counted in the first-digit histogram sh; holders
// counted per attribute of jm and flagged in their position's state byte (pfl: the
// slice's, by list position).  Out of line, so that the register allocation of the
// kernel's other phases does not carry its loads in flight.
template <int D>
__device__ __noinline__ void phase_keys(const float *__restrict__ x, const float *Ls, int d, uint32_t n_live,
                                        uint32_t s0, bool first, bool kc, const uint32_t *sid, const uint32_t *glin,
                                        uint32_t *skey, uint32_t *kpos, uint32_t *sh, uint8_t *pfl, uint32_t *chold,
                                        const uint32_t *jm)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    auto LID = [&](uint32_t q) -> uint32_t { return first ? s0 + q : kc ? sid[q] : __ldcg(&glin[q]); };
    auto key_out = [&](bool live, uint32_t pos, uint32_t k) {
        if (live) {
            if (kc) skey[pos] = k;
            else kpos[pos] = k;
        }
        // the keys of a pass crowd into a few bins: one shared atomic per bin and warp
        const uint32_t b = live ? (k >> 21) : kGone;
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        if (live && lane == __ffs(peers) - 1) atomicAdd(&sh[b], (uint32_t)__popc(peers));
    };
    if constexpr (kCoopRows<D>()) {
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
                uint32_t hz = 0;
#pragma unroll
                for (int u = 0; u < P; u++) {
                    float acc = 0.0f;
                    bool z = false;
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
                        z |= (t0 == 0.0f) | (t1 == 0.0f) | (t2 == 0.0f) | (t3 == 0.0f);
                    }
                    ps[u] = acc;
                    hz |= (uint32_t)z << u;
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
                if (__any_sync(0xffffffffu, hz != 0u)) {
                    // rare: some row of the chunk holds a landmark value (warp-uniform branch)
#pragma unroll 1
                    for (int u = 0; u < P; u++) {
                        const uint32_t id = __shfl_sync(0xffffffffu, myid[q], u * RW + g);
                        const uint32_t rpos = base + q * kThreads + w * 32 + u * RW + g;
                        if (((hz >> u) & 1u) && rpos < n_live) {
                            const float4 *r4 = reinterpret_cast<const float4 *>(x + (size_t)id * D) + sl;
                            for (int f = 0; f < F; f++) {
                                const float4 vv = __ldg(r4 + P * f);
                                const int j = 4 * (sl + P * f);
                                if (vv.x == Ls[j + 0] && in_mask(jm, j + 0)) atomicAdd(&chold[j + 0], 1u);
                                if (vv.y == Ls[j + 1] && in_mask(jm, j + 1)) atomicAdd(&chold[j + 1], 1u);
                                if (vv.z == Ls[j + 2] && in_mask(jm, j + 2)) atomicAdd(&chold[j + 2], 1u);
                                if (vv.w == Ls[j + 3] && in_mask(jm, j + 3)) atomicAdd(&chold[j + 3], 1u);
                            }
                            pfl[rpos] |= kFlHold;
                        }
                    }
                }
                const uint32_t src = (uint32_t)(sl * RW + g);
                const uint32_t pos = base + q * kThreads + w * 32 + src;
                key_out(pos < n_live, pos, __float_as_uint(ps[0]));
            }
        }
    } else {
        constexpr int B = kPeelBatch<D>();
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
            bool hz[B];
#pragma unroll
            for (int q = 0; q < B; q++) dl[q] = dist32<D>(x + (size_t)ids[q] * d, Ls, d, hz[q]);
#pragma unroll
            for (int q = 0; q < B; q++) {
                if (lv[q] && hz[q])
                    note_holder(x + (size_t)ids[q] * d, Ls, d, &pfl[base + q * kThreads + t], chold, jm);
                key_out(lv[q], base + q * kThreads + t, __float_as_uint(dl[q]));
            }
        }
    }
}

// Phase A after a landmark change in the nj attributes jj (ascending; old values jo, new
// values jl): every live key moves by the change of its squared distance,
// sum_i (jl_i - jo_i)(jl_i + jo_i - 2 x_{jj_i}) (FMA chain in float32), read from those
// attributes only; the result is clamped at 0, stored in place and counted in sh, and the
// holders of the new values are counted and flagged as in phase_keys.
template <int D>
__device__ __noinline__ void phase_inc(const float *__restrict__ x, const float *__restrict__ xt, uint32_t n, int d,
                                       uint32_t n_live, bool kc, const uint32_t *sid, const uint32_t *glin,
                                       uint32_t *skey, uint32_t *kpos, uint32_t *sh, uint8_t *pfl, uint32_t *chold,
                                       uint32_t nj, const int *jj, const float *jo, const float *jl)
{
    constexpr int U = 4;                                   // list positions per thread in flight
    const int t = threadIdx.x, lane = t & 31;
    // attribute j of point i at src[i * ps + j * as]: the by-attribute copy (a CTA's ids
    // ascend, so a warp's loads fall close together) or the rows
    const float *src = xt ? xt : x;
    const size_t ps = xt ? 1 : (size_t)(D > 0 ? D : d), as = xt ? (size_t)n : 1;
    for (uint32_t q0 = 0; q0 < n_live; q0 += U * kThreads) {          // block-uniform bound
        uint32_t id[U], key[U], hold = 0;
        float acc[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t qi = q0 + u * kThreads + t;
            const bool v = qi < n_live;
            id[u] = v ? (kc ? sid[qi] : __ldcg(&glin[qi])) : kGone;
            key[u] = v ? (kc ? skey[qi] : __ldcg(&kpos[qi])) : 0u;
            acc[u] = 0.0f;
        }
        for (uint32_t i = 0; i < nj; i++) {
            const int j = jj[i];
            const float ln = jl[i], c = __fsub_rn(ln, jo[i]), sm = __fadd_rn(ln, jo[i]);
            float v[U];
#pragma unroll
            for (int u = 0; u < U; u++) v[u] = id[u] != kGone ? __ldg(&src[(size_t)id[u] * ps + (size_t)j * as]) : ln;
#pragma unroll
            for (int u = 0; u < U; u++) {
                acc[u] = __fmaf_rn(c, __fmaf_rn(-2.0f, v[u], sm), acc[u]);
                if (v[u] == ln && id[u] != kGone) {
                    atomicAdd(&chold[j], 1u);
                    hold |= 1u << u;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t qi = q0 + u * kThreads + t;
            const bool live = id[u] != kGone;
            const float kv = __fadd_rn(__uint_as_float(key[u]), acc[u]);
            const uint32_t k = kv > 0.0f ? __float_as_uint(kv) : 0u;
            if (live) {
                if (kc) skey[qi] = k;
                else kpos[qi] = k;
                if ((hold >> u) & 1u) pfl[qi] |= kFlHold;
            }
            const uint32_t b = live ? (k >> 21) : kGone;
            const uint32_t peers = __match_any_sync(0xffffffffu, b);
            if (live && lane == __ffs(peers) - 1) atomicAdd(&sh[b], (uint32_t)__popc(peers));
        }
    }
}

// A holder's key, as the candidate largest key of each attribute whose landmark value it
// holds.
__device__ __forceinline__ void note_hold_key(const float *__restrict__ row, const float *Ls, int d, uint32_t key,
                                              uint32_t *hmax)
{
    for (int j = 0; j < d; j++)
        if (__ldg(&row[j]) == Ls[j]) atomicMax(&hmax[j], key);
}

// A holder of some attribute's landmark value assigned to round rr of the epoch: counted
// per attribute it holds.
__device__ __forceinline__ void count_holder(const float *__restrict__ x, const float *Ls, int d, uint32_t id,
                                             uint32_t rr, PeelCtl *ctl)
{
    const float *row = x + (size_t)id * d;
    for (int j = 0; j < d; j++)
        if (__ldg(&row[j]) == Ls[j]) atomicAdd(&ctl->hcnt[j][rr], 1u);
}

// Settles group g of the epoch's boundaries (one CTA): every band entry of the group gets
// its round, exactly by (delta64, index).  Entries are ranked by their compensated
// distance; at each boundary only the entries within that distance's error of the cut are
// ranked again by float64.  r0: the epoch's first round; K: its boundaries.
__device__ __noinline__ void settle_group(const PeelArgs &a, const float *Ls, uint32_t g, uint32_t r0, uint32_t K,
                                          uint32_t *scr)
{
    PeelCtl *ctl = a.ctl;
    const int d = a.d;
    const uint32_t N = (uint32_t)a.N;
    const int t = threadIdx.x;
    __shared__ uint32_t s_na;
    __shared__ double s_lo[kMaxEpoch], s_hi[kMaxEpoch];
    __shared__ uint32_t s_need[kMaxEpoch], s_need3[kMaxEpoch], s_na3[kMaxEpoch], s_p3[kMaxEpoch];
    __shared__ unsigned long long s_k3[kMaxEpoch];
    __shared__ uint32_t s_bc[kMaxEpoch];
    const uint32_t q1 = __ldcg(&ctl->g_q1[g]), q2 = __ldcg(&ctl->g_q2[g]);
    const uint32_t ne = __ldcg(&ctl->gcnt[g]);
    // points certainly before the group: certain points of rounds up to q1 and the
    // entries of the groups before it, whose regions precede the group's (q1, g < 32:
    // lane i of warp 0 loads round i's and group i's counts)
    __shared__ uint32_t s_before, s_off;
    if (t < 32) {
        uint32_t cb = (uint32_t)t <= q1 ? __ldcg(&ctl->cert[t]) : 0u;
        uint32_t go = (uint32_t)t < g ? __ldcg(&ctl->gcnt[t]) : 0u;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            cb += __shfl_xor_sync(0xffffffffu, cb, o);
            go += __shfl_xor_sync(0xffffffffu, go, o);
        }
        if (t == 0) {
            s_before = cb + go;
            s_off = go;
        }
    }
    __syncthreads();
    const uint32_t before = s_before, off = s_off;
    const bool staged = ne <= (uint32_t)kStage;
    uint64_t *stk = reinterpret_cast<uint64_t *>(scr + kStageOff);
    uint32_t *stp = scr + kStageOff + 2 * kStage;
    const uint64_t *gk = a.gkey + off;
    const uint32_t *gp = a.gpos + off;
    uint64_t *ak = a.akey + off;
    uint32_t *ap = a.apos + off;
    if (t < kMaxEpoch) s_bc[t] = 0;
    if (t == 0 && __ldcg(&ctl->gfill[g]) != ne) atomicOr(&a.flags[1], 1u);
    if (staged)
        for (uint32_t e = t; e < ne; e += kThreads) {
            stk[e] = __ldcg(&gk[e]);
            stp[e] = __ldcg(&gp[e]);
        }
    __syncthreads();
    auto KA = [&](uint32_t i) -> uint64_t { return staged ? stk[i] : __ldcg(&gk[i]); };
    // an entry's id (bit 31 of the stored word is its hold flag)
    auto PA = [&](uint32_t i) -> uint32_t { return (staged ? stp[i] : __ldcg(&gp[i])) & kPosMask; };
    auto AK = [&](uint32_t i) -> uint64_t { return __ldcg(&ak[i]); };
    auto AP = [&](uint32_t i) -> uint32_t { return __ldcg(&ap[i]); };
    const double win_rel = 4.0 * ((double)eps_ff(d) + 0x1p-52);
    for (uint32_t i = q1; i <= q2; i++) {
        const uint32_t bi = i - q1;
        const int64_t need_s = (int64_t)(i + 1) * N - (int64_t)before;
        uint32_t need = need_s < 0 ? 0u : (need_s > (int64_t)ne ? ne : (uint32_t)need_s);
        if (t == 0 && (need_s < 0 || need_s > (int64_t)ne)) atomicOr(&a.flags[1], 1u);
        if (need == 0 || need == ne) {
            if (t == 0) s_need[bi] = need;
            __syncthreads();
            continue;
        }
        uint64_t V;
        uint32_t Pv;
        select_kth(KA, PA, ne, need, scr, V, Pv);
        const double v = __longlong_as_double((long long)V);
        const double win = win_rel * v + 0x1p-110;
        const double lo = v - win, hi = v + win;
        if (t == 0) s_na = 0;
        __syncthreads();
        uint32_t below = 0;
        for (uint32_t e = t; e < ne; e += kThreads) {
            const double ke = __longlong_as_double((long long)KA(e));
            if (ke < lo) {
                below++;
            } else if (ke <= hi) {
                const uint32_t slot = atomicAdd(&s_na, 1u);
                ap[slot] = PA(e);
            }
        }
        below = block_sum(below);
        const uint32_t na = s_na;
        const uint32_t need3 = need >= below ? need - below : 0u;
        if (t == 0 && (need < below || need3 > na)) atomicOr(&a.flags[1], 1u);
        uint64_t K3 = 0;
        uint32_t P3 = 0;
        if (need3 > 0 && need3 < na) {
            // the entries within the error of the cut-off, ranked by float64 and index
            for (uint32_t e = t; e < na; e += kThreads) {
                const uint32_t pos = __ldcg(&ap[e]);
                ak[e] = (uint64_t)__double_as_longlong(dist64(a.x + (size_t)pos * d, Ls, d));
            }
            __syncthreads();
            select_kth(AK, AP, na, need3, scr, K3, P3);
        }
        if (t == 0) {
            s_need[bi] = need;
            s_lo[bi] = lo;
            s_hi[bi] = hi;
            s_need3[bi] = need3;
            s_na3[bi] = na;
            s_k3[bi] = K3;
            s_p3[bi] = P3;
        }
        __syncthreads();
    }
    // every entry's round: the first boundary of the group plus the boundaries it is after
    for (uint32_t e = t; e < ne; e += kThreads) {
        const uint64_t kb = KA(e);
        const uint32_t raw = staged ? stp[e] : __ldcg(&gp[e]);
        const uint32_t pos = raw & kPosMask;
        const double ke = __longlong_as_double((long long)kb);
        uint32_t after = 0;
        for (uint32_t bi = 0; bi <= q2 - q1; bi++) {
            const uint32_t need = s_need[bi];
            if (need == 0) {
                after++;
                continue;
            }
            if (need == ne || ke < s_lo[bi]) continue;
            if (ke > s_hi[bi]) {
                after++;
                continue;
            }
            const uint32_t n3 = s_need3[bi];
            if (n3 == 0) {
                after++;
            } else if (n3 < s_na3[bi]) {
                const uint64_t k64 = (uint64_t)__double_as_longlong(dist64(a.x + (size_t)pos * d, Ls, d));
                if (k64 > s_k3[bi] || (k64 == s_k3[bi] && pos > s_p3[bi])) after++;
            }
        }
        const uint32_t rr = q1 + after;
        if (rr < K) {
            a.rnd[pos] = r0 + rr;
            atomicAdd(&s_bc[rr], 1u);
            if (raw & ~kPosMask) count_holder(a.x, Ls, d, pos, rr, ctl);
        }
    }
    __syncthreads();
    if (t < (int)K && s_bc[t]) atomicAdd(&ctl->bnd[t], s_bc[t]);
}

// The next landmark (attributes j_first, j_first + j_step, ...): in each attribute the
// smallest value among the points left (rnd >= live_from), found from the bucket order:
// from the attribute's bucket pointer on, the first bucket whose entries include a point
// left holds it.  A point taken stays taken (live_from only grows), so each bucket's start
// is moved past the entries found gone and a bucket whose start reaches its end is passed
// for good: every entry is found gone at most once per run.  Buckets are examined kThreads
// at a time, a thread peeking at the next kPeek entries of its bucket (their loads issued
// together); a bucket that still has entries after those, and the first bucket with a
// point left, are scanned by the whole CTA.
constexpr int kPeek = 16;

__device__ __noinline__ void find_landmark(const PeelArgs &a, int j_first, int j_step, uint32_t live_from)
{
    PeelCtl *ctl = a.ctl;
    const int d = a.d;
    const uint32_t nbk = a.nbk;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    __shared__ uint32_t red_a[kW], red_u[kW], red_b[kW], red_p[kW];
    __shared__ uint32_t s_st, s_en;
    for (int j = j_first; j >= 0 && j < d; j += j_step) {
        uint4 *bj = a.bcs + (size_t)j * nbk;
        const uint32_t *oj = a.ord + (size_t)j * a.ord_ld;
        uint32_t b = __ldcg(&ctl->lptr[j]);       // the buckets before b hold no point left
        uint32_t mnb = kGone;
        while (b < nbk) {
            // bucket b + t: 1 = a point left among its next kPeek entries, 2 = entries left
            // to look at after those, 0 = nothing left
            const uint32_t bb = b + (uint32_t)t;
            uint4 e = bb < nbk ? __ldcg(&bj[bb]) : make_uint4(0u, 0u, 0u, 0u);
            int state = 0;
            if (e.y < e.z) {
                uint32_t ids[kPeek];
#pragma unroll
                for (int i = 0; i < kPeek; i++) ids[i] = e.y + i < e.z ? __ldcg(&oj[e.y + i]) : kGone;
                uint32_t first = kPeek;
#pragma unroll
                for (int i = kPeek - 1; i >= 0; i--)
                    if (ids[i] != kGone && __ldcg(&a.rnd[ids[i]]) >= live_from) first = (uint32_t)i;
                const uint32_t adv = first < kPeek ? first : min((uint32_t)kPeek, e.z - e.y);
                if (adv) {
                    e.y += adv;
                    reinterpret_cast<uint32_t *>(&bj[bb])[1] = e.y;     // entries before e.y are gone
                }
                state = first < kPeek ? 1 : (e.y < e.z ? 2 : 0);
            }
            uint32_t fa = warp_min(state == 1 ? bb : kGone), fu = warp_min(state == 2 ? bb : kGone);
            if (lane == 0) {
                red_a[w] = fa;
                red_u[w] = fu;
            }
            __syncthreads();
            fa = red_a[0];
            fu = red_u[0];
#pragma unroll
            for (int q = 1; q < kW; q++) {
                fa = min(fa, red_a[q]);
                fu = min(fu, red_u[q]);
            }
            const uint32_t fb = min(fa, fu);
            if (bb == fb) {
                s_st = e.y;
                s_en = e.z;
            }
            __syncthreads();
            if (fb == kGone) {                     // kThreads buckets with nothing left
                b += kThreads;
                continue;
            }
            // bucket fb, the whole CTA: the smallest value among its entries left and the
            // first of them (its start moves there, or to its end)
            const uint32_t st = s_st, en = s_en;
            uint32_t lm = kGone, fp = en;
            for (uint32_t q = st + t; q < en; q += kThreads) {
                const uint32_t id = __ldcg(&oj[q]);
                if (__ldcg(&a.rnd[id]) >= live_from) {
                    lm = min(lm, __float_as_uint(__ldg(&a.x[(size_t)id * d + j])));
                    fp = min(fp, q);
                }
            }
            lm = warp_min(lm);
            fp = warp_min(fp);
            if (lane == 0) {
                red_b[w] = lm;
                red_p[w] = fp;
            }
            __syncthreads();
            lm = red_b[0];
            fp = red_p[0];
#pragma unroll
            for (int q = 1; q < kW; q++) {
                lm = min(lm, red_b[q]);
                fp = min(fp, red_p[q]);
            }
            if (t == 0 && fp > st) reinterpret_cast<uint32_t *>(&bj[fb])[1] = fp;
            __syncthreads();
            if (lm != kGone) {
                mnb = lm;
                b = fb;
                break;
            }
            b = fb + 1;                            // every entry of fb is gone
        }
        if (t == 0) {
            const uint32_t nb = mnb == kGone ? kInfBits : mnb;
            ctl->lptr[j] = b;
            if (nb != __ldcg(&ctl->Lbits[j])) ctl->chold[j] = 0;    // a new value: its holders are counted again
            ctl->Lbits[j] = nb;
        }
    }
}

// The last CTA of phase B turns each boundary's first-digit bin and rank inside it into
// its band cut-offs (second digit from the boundary's histogram), and merges boundaries
// whose bands overlap into groups.  Warp w resolves boundaries w, w + kW, ...: lane i sums
// second-digit bins [64 i, 64 i + 64) in two halves, a warp scan finds the lane holding
// the rank, and that lane walks the half holding it (its loads issued together).
__device__ __noinline__ void resolve_cutoffs(PeelCtl *ctl, uint32_t Kb, uint32_t N, int d, float keps, float kabs,
                                             const uint32_t *sb, const uint32_t *sr, const uint32_t *sslot,
                                             const uint32_t *sbin, uint32_t nslot)
{
    __shared__ uint32_t s_b1[kMaxEpoch];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t < kMaxEpoch) s_b1[t] = 0;
    // the rounds this landmark can serve: up to the one in which the last holder of some
    // attribute's landmark value leaves (the landmark changes after it).  That holder's key
    // m (the smallest over the attributes of their holders' largest key) is at most the
    // c-th smallest live key, c read off the histograms (the second digit where m's bin has
    // one), so it leaves at the latest in round (c - 1) / N; the boundaries past that
    // round are not resolved (a prediction that falls short costs one more epoch)
    uint32_t m = kGone;
    for (int j = t; j < d; j += kThreads) m = min(m, __ldcg(&ctl->hmax[j]));
    m = block_min(m);
    const uint32_t mb0 = m >> 21, mb1 = (m >> 10) & (kHistBins - 1);
    int slot = -1;
    for (uint32_t q = 0; q < nslot; q++)
        if (sbin[q] == mb0) slot = (int)q;
    uint32_t cnt = 0;
    for (int b = t; b < kHistBins; b += kThreads) {
        if ((uint32_t)b < mb0 || ((uint32_t)b == mb0 && slot < 0)) cnt += __ldcg(&ctl->h0[b]);
        if (slot >= 0 && (uint32_t)b <= mb1) cnt += __ldcg(&ctl->h1[slot][b]);
    }
    cnt = block_sum(cnt);
    const uint32_t K = min(Kb, (cnt > 0 ? (cnt - 1) / N : 0u) + 1u);
    __syncthreads();
    for (uint32_t q = (uint32_t)w; q < K; q += kW) {
        const uint4 *h4 = reinterpret_cast<const uint4 *>(ctl->h1[sslot[q]] + lane * 64);
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const uint4 u = __ldcg(h4 + i), v = __ldcg(h4 + 8 + i);
            lo += u.x + u.y + u.z + u.w;
            hi += v.x + v.y + v.z + v.w;
        }
        const uint32_t ls = lo + hi;
        const uint32_t ex = warp_incl_scan(ls) - ls;
        const uint32_t r = sr[q];
        if (r >= ex && r < ex + ls) {
            const int half = r >= ex + lo ? 1 : 0;
            uint4 u[8];
#pragma unroll
            for (int i = 0; i < 8; i++) u[i] = __ldcg(h4 + 8 * half + i);
            uint32_t cc = ex + (half ? lo : 0u), found = 0;
            bool done = false;
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const uint32_t v4[4] = {u[i].x, u[i].y, u[i].z, u[i].w};
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (!done && r < cc + v4[k]) {
                        found = (uint32_t)(lane * 64 + 32 * half + 4 * i + k);
                        done = true;
                    }
                    cc += v4[k];
                }
            }
            s_b1[q] = found;
        }
    }
    __syncthreads();
    if (t == 0) {
        uint32_t ng = 0, gi = 0, go = 0;
        for (uint32_t q = 0; q < K; q++) {
            uint32_t ik, ok;
            band_cutoffs(sb[q], s_b1[q], keps, kabs, ik, ok);
            if (ng > 0 && ik <= go) {
                go = max(go, ok);
                ctl->g_out[ng - 1] = go;
                ctl->g_q2[ng - 1] = q;
            } else {
                gi = ik;
                go = ok;
                ctl->g_in[ng] = gi;
                ctl->g_out[ng] = go;
                ctl->g_q1[ng] = q;
                ctl->g_q2[ng] = q;
                ng++;
            }
        }
        ctl->n_groups = ng;
        ctl->n_slots = nslot;
        ctl->k_eff = K;
        ctl->kref = __uint_as_float(sb[0] << 21);
    }
}

// The last CTA of phase D finds how many rounds the epoch commits: up to the first round
// after which some attribute has no holder of its landmark value left (the landmark then
// changes).  It updates the live holder counts, checks that every round of the epoch got
// exactly N points, records the epoch's landmarks and publishes k_commit and l_changed.
__device__ __noinline__ void commit_count(const PeelArgs &a, const float *Ls, uint32_t K, uint32_t r0, bool need_keys)
{
    PeelCtl *ctl = a.ctl;
    const int d = a.d;
    const uint32_t N = (uint32_t)a.N;
    const int t = threadIdx.x;
    // per attribute: the first round after which no holder of L_j is left
    // (the counts are read all at once, then scanned in registers)
    uint32_t qs = kNone;
    for (int j = t; j < d; j += kThreads) {
        uint32_t hc[kMaxEpoch];
#pragma unroll
        for (int r = 0; r < kMaxEpoch; r++) hc[r] = r < (int)K ? __ldcg(&ctl->hcnt[j][r]) : 0u;
        const uint32_t ch = __ldcg(&ctl->chold[j]);
        uint32_t acc = 0, qj = kNone;
#pragma unroll
        for (int r = 0; r < kMaxEpoch; r++) {
            acc += hc[r];
            if (qj == kNone && r < (int)K && acc >= ch) qj = (uint32_t)r;
        }
        qs = min(qs, qj);
    }
    qs = block_min(qs);
    const uint32_t kc_ = qs < K ? qs + 1u : K;
    const bool changed = qs < K;
    // the holders that leave with the committed rounds (an attribute whose landmark value
    // changes has its count cleared by find_landmark and counted again by the next pass)
    for (int j = t; j < d; j += kThreads) {
        uint32_t gone = 0;
#pragma unroll
        for (int r = 0; r < kMaxEpoch; r++) gone += r < (int)kc_ ? __ldcg(&ctl->hcnt[j][r]) : 0u;
        ctl->chold[j] = __ldcg(&ctl->chold[j]) - gone;
    }
    if (t < (int)K && __ldcg(&ctl->cert[t]) + __ldcg(&ctl->bnd[t]) != N) atomicOr(&a.flags[1], 1u);
    if (changed) {
        for (int b = t; b < kHistBins; b += kThreads) ctl->h0[b] = 0;
        for (int j = t; j < d; j += kThreads) ctl->hmax[j] = 0;    // recomputed by the next pass
    }
    if (a.landmarks)
        for (uint32_t e = t; e < kc_ * (uint32_t)d; e += kThreads)
            a.landmarks[(size_t)(r0 + e / d) * d + e % d] = Ls[e % d];
    if (t == 0) {
        ctl->k_commit = kc_;
        ctl->l_changed = changed ? 1u : 0u;
        ctl->epochs += 1;
        ctl->passes += need_keys ? 1u : 0u;
    }
}

// A CTA's list of points left, by list position: ids, float32 keys and state bytes; in
// shared memory when the slice fits the key cache (kc), else in one of two global lists.
struct ListView {
    bool first, kc;
    uint32_t s0;
    const uint32_t *sid, *skey;
    uint8_t *sfl;
    const uint32_t *gid, *gkp;
    uint8_t *gfl;
    uint32_t *gid2, *gkp2;       // the other global list (compaction target)
    uint8_t *gfl2;
    __device__ __forceinline__ uint32_t id(uint32_t q) const { return first ? s0 + q : kc ? sid[q] : __ldcg(&gid[q]); }
    __device__ __forceinline__ uint32_t key(uint32_t q) const { return kc ? skey[q] : __ldcg(&gkp[q]); }
    __device__ __forceinline__ uint8_t *fl() const { return kc ? sfl : gfl; }
};

// Phase C for one CTA's list: every live key classified against the epoch's groups (see
// the kernel); certain points get their round in rnd[] and counted in s_cc, band entries
// are listed (with their hold flag in bit 31 of the id) and counted per group in s_gc.
__device__ __noinline__ void classify_live(const PeelArgs &a, const ListView &L, uint32_t n_live, const float *Ls,
                                          uint32_t r0, uint32_t K, uint32_t ng, const uint32_t *s_gin,
                                          const uint32_t *s_gout, const uint32_t *s_gq2, uint32_t s_glast,
                                          uint32_t *s_cc, uint32_t *s_gc)
{
    PeelCtl *ctl = a.ctl;
    const int d = a.d;
    const int t = threadIdx.x, lane = t & 31;
    const uint32_t lt = (1u << lane) - 1u;
    uint8_t *pfl = L.fl();
    // a key's class: kNone (after the epoch, or past the end of the list), its round r < K
    // (certainly), or kBandTag | g (in group g's band).  The keys, ids and state bytes of
    // kCB positions are loaded before any is used; the class goes to the state byte and is
    // counted in shared memory (the points of the epoch are spread over the list, so few
    // lanes of a warp meet on one counter).
    constexpr uint32_t kBandTag = 0x100u;
    for (uint32_t q0 = 0; q0 < n_live; q0 += kCB * kThreads) {
        uint32_t kk[kCB], cls[kCB], idv[kCB], fl[kCB];
#pragma unroll
        for (int u = 0; u < kCB; u++) {
            const uint32_t qi = q0 + u * kThreads + t;
            const bool v = qi < n_live;
            kk[u] = v ? L.key(qi) : kGone;
            idv[u] = v ? L.id(qi) : 0u;
            fl[u] = v ? pfl[qi] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kCB; u++) {
            cls[u] = kNone;
            if (kk[u] <= s_glast) {
                uint32_t g = 0, cum = 0;
                while (g < ng && kk[u] > s_gout[g]) {
                    cum = s_gq2[g] + 1u;
                    g++;
                }
                if (g < ng && kk[u] >= s_gin[g]) cls[u] = kBandTag | g;
                else if (cum < K) cls[u] = cum;
            }
            // a point outside the epoch keeps its state byte (kFlNone since the last commit)
            if (cls[u] != kNone)
                pfl[q0 + u * kThreads + t] = (uint8_t)((fl[u] & kFlHold) | (cls[u] >= kBandTag ? kFlBand : cls[u]));
        }
#pragma unroll
        for (int u = 0; u < kCB; u++) {
            const bool band = cls[u] != kNone && cls[u] >= kBandTag;
            const bool cert = cls[u] < kBandTag;
            const uint32_t bm = __ballot_sync(0xffffffffu, band);
            if (bm) {
                uint32_t base = 0;
                const int leader = __ffs(bm) - 1;
                if (lane == leader) base = atomicAdd(&ctl->band_cnt, (uint32_t)__popc(bm));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (band) {
                    const uint32_t slot = base + (uint32_t)__popc(bm & lt);
                    a.band_k32[slot] = kk[u];
                    a.band_pos[slot] = idv[u] | ((fl[u] & kFlHold) ? ~kPosMask : 0u);
                    atomicAdd(&s_gc[cls[u] - kBandTag], 1u);
                }
            }
            if (cert) {
                a.rnd[idv[u]] = r0 + cls[u];
                atomicAdd(&s_cc[cls[u]], 1u);
                if (fl[u] & kFlHold) count_holder(a.x, Ls, d, idv[u], cls[u], ctl);
            }
        }
    }
}

// Phase E for a list in shared memory (kc), compacted in place: the points whose round
// lies before live_from leave it; dropped assignments are reset; with the landmark kept,
// the committed keys leave the first-digit histogram.  Returns the points left.
__device__ __noinline__ uint32_t compact_shared(const PeelArgs &a, const ListView &L, uint32_t n_live, uint32_t r0,
                                                uint32_t live_from, bool changed, uint32_t *scr)
{
    PeelCtl *ctl = a.ctl;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    uint8_t *pfl = L.sfl;
    if (!changed)
        for (int b = t; b < kHistBins; b += kThreads) scr[b] = 0;
    __syncthreads();
    constexpr int PER = kQT * kW / 32;
    static_assert(PER * 32 == kQT * kW, "one warp scans the tile counts");
    __shared__ uint32_t woff[kQT * kW + 1];
    uint32_t *kid = const_cast<uint32_t *>(L.sid), *kkey = const_cast<uint32_t *>(L.skey);
    uint32_t done = 0;
    // in place: a tile's ids, keys and state bytes are all read before any kept one
    // is written, and those land at or below the tile's own positions.  A position's
    // state byte tells its round in the epoch; only band entries read their round
    // (settled by another CTA) from rnd[].
    for (uint32_t cb = 0; cb < n_live; cb += kQT * kThreads) {
        uint32_t ids[kQT], keys[kQT], fls[kQT], rv[kQT], vl = 0, kp = 0;
#pragma unroll
        for (int q = 0; q < kQT; q++) {
            const uint32_t qi = cb + q * kThreads + t;
            const bool v = qi < n_live;
            ids[q] = v ? L.id(qi) : 0u;
            keys[q] = v ? L.key(qi) : kGone;
            fls[q] = v ? pfl[qi] : (uint32_t)kFlNone;
            vl |= (uint32_t)v << q;
        }
#pragma unroll
        for (int q = 0; q < kQT; q++) {
            const uint32_t st = fls[q] & 0x7Fu;
            rv[q] = st == kFlBand ? __ldcg(&a.rnd[ids[q]]) : st == kFlNone ? kNone : r0 + st;
            kp |= (uint32_t)(((vl >> q) & 1u) && rv[q] >= live_from) << q;
        }
        uint32_t bk[kQT];
#pragma unroll
        for (int q = 0; q < kQT; q++) {
            bk[q] = __ballot_sync(0xffffffffu, (kp >> q) & 1u);
            if (lane == 0) woff[q * kW + w] = __popc(bk[q]);
        }
        __syncthreads();
        if (w == 0) {
            uint32_t vk[PER], sk = 0;
#pragma unroll
            for (int e = 0; e < PER; e++) {
                vk[e] = woff[lane * PER + e];
                sk += vk[e];
            }
            const uint32_t ik = warp_incl_scan(sk);
            uint32_t ek = ik - sk;
#pragma unroll
            for (int e = 0; e < PER; e++) {
                woff[lane * PER + e] = ek;
                ek += vk[e];
            }
            if (lane == 31) woff[kQT * kW] = ik;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kQT; q++) {
            const bool valid = (vl >> q) & 1u;
            const bool keep = (kp >> q) & 1u;
            if (keep) {
                const uint32_t o = done + woff[q * kW + w] + __popc(bk[q] & lt);
                kid[o] = ids[q];
                kkey[o] = keys[q];
                pfl[o] = (uint8_t)((fls[q] & kFlHold) | kFlNone);
                if (rv[q] != kNone) a.rnd[ids[q]] = kNone;       // an assignment dropped
            } else if (valid && !changed) {
                // the next epoch keeps these keys: the committed ones leave the histogram
                atomicAdd(&scr[keys[q] >> 21], 1u);
            }
        }
        done += woff[kQT * kW];
        __syncthreads();
    }

    if (!changed) {
        // the next epoch keeps these keys: the committed ones leave the histogram
        __syncthreads();
        for (int b = t; b < kHistBins; b += kThreads)
            if (scr[b]) atomicSub(&ctl->h0[b], scr[b]);
    }
    return done;
}

// Phase E for a list in global memory: each warp takes chunks of 32 kQT positions and
// appends the points it keeps to the other list (their order does not matter: the
// subclusters are packed by a counting sort over rnd afterwards), claiming slots with one
// shared atomic per 32 positions; no block barrier inside.  Returns the points left.
__device__ __noinline__ uint32_t compact_global(const PeelArgs &a, const ListView &L, uint32_t n_live, uint32_t r0,
                                                uint32_t live_from, bool changed, uint32_t *scr)
{
    PeelCtl *ctl = a.ctl;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    __shared__ uint32_t s_out;
    if (!changed)
        for (int b = t; b < kHistBins; b += kThreads) scr[b] = 0;
    if (t == 0) s_out = 0;
    __syncthreads();
    for (uint32_t cb = (uint32_t)w * 32 * kQT; cb < n_live; cb += kW * 32 * kQT) {
        uint32_t ids[kQT], keys[kQT], fls[kQT];
#pragma unroll
        for (int q = 0; q < kQT; q++) {
            const uint32_t qi = cb + q * 32 + lane;
            const bool v = qi < n_live;
            ids[q] = v ? L.id(qi) : 0u;
            keys[q] = v ? __ldcg(&L.gkp[qi]) : kGone;
            fls[q] = v ? L.gfl[qi] : (uint32_t)kFlNone;
        }
        uint32_t bk[kQT], rvs[kQT], tot = 0;
#pragma unroll
        for (int q = 0; q < kQT; q++) {
            const bool valid = cb + q * 32 + lane < n_live;
            const uint32_t st = fls[q] & 0x7Fu;
            rvs[q] = st == kFlBand ? __ldcg(&a.rnd[ids[q]]) : st == kFlNone ? kNone : r0 + st;
            bk[q] = __ballot_sync(0xffffffffu, valid && rvs[q] >= live_from);
            tot += __popc(bk[q]);
        }
        // one slot claim per warp and chunk
        uint32_t ob = 0;
        if (lane == 0 && tot) ob = atomicAdd(&s_out, tot);
        ob = __shfl_sync(0xffffffffu, ob, 0);
#pragma unroll
        for (int q = 0; q < kQT; q++) {
            const bool valid = cb + q * 32 + lane < n_live;
            if ((bk[q] >> lane) & 1u) {
                const uint32_t o = ob + __popc(bk[q] & lt);
                L.gid2[o] = ids[q];
                L.gkp2[o] = keys[q];
                L.gfl2[o] = (uint8_t)((fls[q] & kFlHold) | kFlNone);
                if (rvs[q] != kNone) a.rnd[ids[q]] = kNone;          // an assignment dropped
            } else if (valid && !changed) {
                atomicAdd(&scr[keys[q] >> 21], 1u);
            }
            ob += __popc(bk[q]);
        }
    }
    __syncthreads();
    if (!changed) {
        // the next epoch keeps these keys: the committed ones leave the histogram
        __syncthreads();
        for (int b = t; b < kHistBins; b += kThreads)
            if (scr[b]) atomicSub(&ctl->h0[b], scr[b]);
    }
    return s_out;
}

template <int D>
__global__ void __launch_bounds__(kThreads) k_peel(PeelArgs a)
{
    // dynamic shared memory: [scratch: phase A's histogram | selection scratch + staged
    // band entries] [keys by list position | ids by list position] (the latter when kc)
    extern __shared__ __align__(16) uint32_t dyn[];
    uint32_t *scr = dyn;
    uint32_t *skey = dyn + kScrWords;
    uint32_t *sid = skey + kKeyCache;
    uint8_t *sfl = reinterpret_cast<uint8_t *>(sid + kKeyCache);     // state bytes by list position (kc)
    __shared__ float Ls[D > 0 ? D : kMaxD];
    __shared__ uint32_t s_b[kMaxEpoch], s_r[kMaxEpoch], s_slot[kMaxEpoch], s_sbin[kMaxEpoch];
    __shared__ uint32_t s_gin[kMaxEpoch], s_gout[kMaxEpoch], s_gq2[kMaxEpoch];
    __shared__ uint32_t s_cc[kMaxEpoch], s_gc[kMaxEpoch];
    __shared__ uint32_t s_nslot, s_glast;
    __shared__ uint8_t s_map[kHistBins];
    // the previous epoch's landmark; the attributes whose landmark value is new (mask) and,
    // for an update of the keys, those attributes with their old and new values
    __shared__ float Lold[D > 0 ? D : kMaxD];
    __shared__ uint32_t s_jm[kMaxD / 32];
    __shared__ int s_ij[kIncMax];
    __shared__ float s_io[kIncMax], s_il[kIncMax];
    __shared__ uint32_t s_nj;
    __shared__ int s_inc;
    __shared__ float s_keps, s_kabs;
    PeelCtl *ctl = a.ctl;
    const int d = a.d;
    const uint32_t n = (uint32_t)a.n, N = (uint32_t)a.N;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const unsigned G = gridDim.x, c = blockIdx.x;
    const unsigned lim = a.spin;
    // With 16 CTAs or more, the last Gl CTAs own no points and only build landmarks, which
    // then overlaps with the others' compaction; otherwise every CTA does both.
    const int Gl = G >= 16 ? min(d, (int)(G / 8)) : 0;
    const unsigned Gs = G - (unsigned)Gl;
    const uint32_t s0 = c < Gs ? (uint32_t)((uint64_t)c * n / Gs) : n;
    const uint32_t s1 = c < Gs ? (uint32_t)((uint64_t)(c + 1) * n / Gs) : n;
    const int lm_first = Gl ? (int)c - (int)Gs : (int)(G - 1 - c);
    const int lm_step = Gl ? Gl : (int)G;
    uint32_t n_live = s1 - s0;           // points of the slice left
    const bool kc = s1 - s0 <= (uint32_t)kKeyCache;   // the list and its keys stay in shared memory
    // slices beyond the key cache alternate between two lists in global memory
    uint32_t *gid = a.lidx + s0, *gid2 = a.lidx + n + s0;
    uint32_t *gkp = a.kpos + s0, *gkp2 = a.kpos + n + s0;
    uint8_t *gfl = a.pflag + s0, *gfl2 = a.pflag + n + s0;
    uint8_t *pfl = kc ? sfl : gfl;                      // the slice's state bytes by list position
    unsigned gen = 0;
    if (kc)
        for (uint32_t q = t; q < s1 - s0; q += kThreads) sfl[q] = kFlNone;

    // ---- before the first epoch: per attribute, the point ids by value bucket (counting sort)
    // The attributes go in groups of kBkGroup, each group one grid-stride sweep over its
    // (point, attribute) pairs, kBkUnroll pairs per thread at a time (their loads, then
    // their atomics, then their stores, so that each thread keeps several of each in
    // flight).  A sweep writes the lists through kBkGroup x nbk cursors, few enough that
    // the partly written sectors at the cursors stay in L2 until they fill.
    {
        const uint32_t nbk = a.nbk;
        const uint32_t stride = G * (uint32_t)kThreads;
        const uint32_t e0 = c * (uint32_t)kThreads + (uint32_t)t;
        for (int pass = 0; pass < 2; pass++) {
            for (int j0 = 0; j0 < d; j0 += kBkGroup) {
                const uint32_t w = (uint32_t)min(kBkGroup, d - j0);
                const uint32_t si = stride / w, sj = stride % w;
                uint32_t i = e0 / w, j = e0 % w;
                while (i < n) {
                    uint32_t pi[kBkUnroll], pj[kBkUnroll], pb[kBkUnroll];
#pragma unroll
                    for (int u = 0; u < kBkUnroll; u++) {
                        pi[u] = i;
                        pj[u] = (uint32_t)j0 + j;
                        pb[u] = i < n ? bucket_of(__ldg(&a.x[(size_t)i * d + j0 + j]), nbk) : 0u;
                        i += si;
                        j += sj;
                        if (j >= w) {
                            j -= w;
                            i++;
                        }
                    }
                    if (pass == 0) {
#pragma unroll
                        for (int u = 0; u < kBkUnroll; u++)
                            if (pi[u] < n) atomicAdd(&a.bcnt[(size_t)pj[u] * nbk + pb[u]], 1u);
                    } else {
#pragma unroll
                        for (int u = 0; u < kBkUnroll; u++)
                            if (pi[u] < n) pb[u] = atomicAdd(&a.bcnt[(size_t)pj[u] * nbk + pb[u]], 1u);
#pragma unroll
                        for (int u = 0; u < kBkUnroll; u++)
                            if (pi[u] < n) a.ord[(size_t)pj[u] * a.ord_ld + pb[u]] = pi[u];
                    }
                }
            }
            if (!grid_sync(ctl, a.flags, gen, lim, pass == 0 ? a.stall : 0u)) return;
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
            if (!grid_sync(ctl, a.flags, gen, lim)) return;
        }
    }

    bool first = true;           // the first epoch: a slice's list is the slice itself
    bool need_keys = true;       // the landmark changed: the keys must be computed
    uint32_t r0 = 0;             // the epoch's first round
    // the keys' error bound |delta32 - delta64| <= k_eps delta32 + k_abs (thread 0 keeps it,
    // the same in every CTA) and the key updates since the last full pass
    const double eps0 = (double)(d + 4) * 0x1p-23;
    double k_eps = eps0, k_abs = 0x1p-120;
    for (;;) {
        const uint32_t nl_tot = n - r0 * N;
        auto LID = [&](uint32_t q) -> uint32_t { return first ? s0 + q : kc ? sid[q] : __ldcg(&gid[q]); };
        auto LKEY = [&](uint32_t q) -> uint32_t { return kc ? skey[q] : __ldcg(&gkp[q]); };
        const ListView LV{first, kc, s0, sid, skey, sfl, gid, gkp, gfl, gid2, gkp2, gfl2};
        for (int j = t; j < d; j += kThreads) {
            Lold[j] = Ls[j];
            Ls[j] = __uint_as_float(__ldcg(&ctl->Lbits[j]));
        }
        __syncthreads();
        if (nl_tot <= N) {                            // the last subcluster: all that is left
            for (uint32_t q = t; q < n_live; q += kThreads) a.rnd[LID(q)] = r0;
            if (c == 0 && a.landmarks)
                for (int j = t; j < d; j += kThreads) a.landmarks[(size_t)r0 * d + j] = Ls[j];
            break;
        }
        const uint32_t Kb = min(a.kmax, (nl_tot + N - 1) / N - 1u);   // boundaries phase B locates

        // ---- A: float32 distances of the points left, the first histogram, the holders
        if (need_keys) {
            // the attributes whose landmark value is new (all of them at first)
            for (int j0 = w * 32; j0 < d; j0 += kW * 32) {
                const int j = j0 + lane;
                const bool mv = j < d && (first || __float_as_uint(Ls[j]) != __float_as_uint(Lold[j]));
                const uint32_t m = __ballot_sync(0xffffffffu, mv);
                if (lane == 0) s_jm[j0 >> 5] = m;
            }
            for (int b = t; b < kHistBins; b += kThreads) scr[b] = 0;
            __syncthreads();
            if (t == 0) {
                // an update of the keys, or a full pass (the same choice in every CTA)
                uint32_t nj = 0, nsec = 0, last_sec = kGone;
                double cs = 0.0;
                bool fin = true;
                for (int wd = 0; wd < (d + 31) / 32; wd++) {
                    uint32_t m = s_jm[wd];
                    while (m) {
                        const int j = wd * 32 + __ffs(m) - 1;
                        m &= m - 1u;
                        if (nj < (uint32_t)kIncMax) {
                            s_ij[nj] = j;
                            s_io[nj] = Lold[j];
                            s_il[nj] = Ls[j];
                            const float c = __fsub_rn(Ls[j], Lold[j]);
                            fin = fin && c >= 0.0f && c <= 1.0f;
                            cs += (double)c;
                        }
                        nj++;
                        if ((uint32_t)(j >> 3) != last_sec) {
                            nsec++;
                            last_sec = (uint32_t)(j >> 3);
                        }
                    }
                }
                const double ne = k_eps + 0x1p-23;
                const double na = k_abs + (5.0 * k_eps + (16.0 + 4.0 * nj) * 0x1p-24) * cs * (1.0 + 0x1p-20);
                // the absolute term stays below an eighth of the relative one at the last
                // epoch's first boundary, so the bands widen little
                const double kref = (double)__ldcg(&ctl->kref);
                const bool inc = !first && fin && nj >= 1 && nj <= (uint32_t)kIncMax && nsec * 160u < 12u * (uint32_t)d &&
                                 ne <= 1.5 * eps0 && na <= 0.125 * eps0 * kref;
                if (inc) {
                    k_eps = ne;
                    k_abs = na;
                } else {
                    k_eps = eps0;
                    k_abs = 0x1p-120;
                }
                s_nj = inc ? nj : 0u;
                s_inc = inc ? 1 : 0;
                if (inc && c == 0) ctl->key_updates += 1;
                s_keps = __double2float_ru(k_eps);
                s_kabs = __double2float_ru(k_abs);
            }
            __syncthreads();
            if (s_inc)
                phase_inc<D>(a.x, a.xt, n, d, n_live, kc, sid, gid, skey, gkp, scr, pfl, ctl->chold, s_nj, s_ij, s_io,
                             s_il);
            else
                phase_keys<D>(a.x, Ls, d, n_live, s0, first, kc, sid, gid, skey, gkp, scr, pfl, ctl->chold, s_jm);
            __syncthreads();
            // each attribute's largest holder key (the holders are the flagged points left)
            for (uint32_t q0 = 0; q0 < n_live; q0 += kHoldBatch * kThreads) {
                uint8_t f[kHoldBatch];
#pragma unroll
                for (int u = 0; u < kHoldBatch; u++) {
                    const uint32_t qi = q0 + u * kThreads + t;
                    f[u] = qi < n_live ? pfl[qi] : (uint8_t)0;
                }
#pragma unroll
                for (int u = 0; u < kHoldBatch; u++)
                    if (f[u] & kFlHold) {
                        const uint32_t qi = q0 + u * kThreads + t;
                        note_hold_key(a.x + (size_t)LID(qi) * d, Ls, d, LKEY(qi), ctl->hmax);
                    }
            }
            for (int b = t; b < kHistBins; b += kThreads)
                if (scr[b]) atomicAdd(&ctl->h0[b], scr[b]);
            if (!grid_sync(ctl, a.flags, gen, lim)) return;
        }

        // ---- B: each boundary's first-digit bin (every CTA), then second-digit histograms
        {
            constexpr int per = kHistBins / kThreads;       // 8 bins per thread
            uint32_t l0[per];
            const uint4 *p = reinterpret_cast<const uint4 *>(ctl->h0 + t * per);
            const uint4 u = __ldcg(p), v = __ldcg(p + 1);
            l0[0] = u.x; l0[1] = u.y; l0[2] = u.z; l0[3] = u.w;
            l0[4] = v.x; l0[5] = v.y; l0[6] = v.z; l0[7] = v.w;
            uint32_t s = 0;
#pragma unroll
            for (int q = 0; q < per; q++) s += l0[q];
            uint32_t tot;
            const uint32_t e0 = block_excl_scan(s, tot);
            for (uint32_t q = 0; q < Kb; q++) {
                const uint32_t target = (q + 1) * N - 1u;
                if (target >= e0 && target < e0 + s) {
                    uint32_t cc = e0;
#pragma unroll
                    for (int i = 0; i < per; i++) {
                        if (target >= cc && target < cc + l0[i]) {
                            s_b[q] = (uint32_t)(t * per + i);
                            s_r[q] = target - cc;
                        }
                        cc += l0[i];
                    }
                }
            }
            for (int b = t; b < kHistBins; b += kThreads) s_map[b] = 0xFF;
            __syncthreads();
            if (t == 0) {
                uint32_t ns = 0;
                for (uint32_t q = 0; q < Kb; q++) {
                    if (q == 0 || s_b[q] != s_b[q - 1]) s_sbin[ns++] = s_b[q];
                    s_slot[q] = ns - 1;
                }
                s_nslot = ns;
                if (tot != nl_tot) atomicOr(&a.flags[1], 1u);
            }
            __syncthreads();
            if (t < (int)s_nslot) s_map[s_sbin[t]] = (uint8_t)t;
            __syncthreads();
            // in shared memory for the first kSlotsSmem bins (the others straight to global),
            // then the non-zero bins added to the grid's histograms
            const uint32_t nss = min(s_nslot, (uint32_t)kSlotsSmem);
            for (uint32_t b = t; b < nss * kHistBins; b += kThreads) scr[b] = 0;
            __syncthreads();
            for (uint32_t q0 = t; q0 < n_live; q0 += 4 * kThreads) {
                uint32_t k4[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t qi = q0 + q * kThreads;
                    k4[q] = qi < n_live ? LKEY(qi) : kGone;
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t sl = k4[q] == kGone ? 0xFFu : s_map[k4[q] >> 21];
                    const uint32_t sub = (k4[q] >> 10) & (kHistBins - 1);
                    if (sl < nss) atomicAdd(&scr[sl * kHistBins + sub], 1u);
                    else if (sl != 0xFFu) atomicAdd(&ctl->h1[sl][sub], 1u);
                }
            }
            __syncthreads();
            for (uint32_t b = t; b < nss * kHistBins; b += kThreads)
                if (scr[b]) atomicAdd(&ctl->h1[b / kHistBins][b % kHistBins], scr[b]);
        }
        // the last CTA to arrive turns each boundary's bins into its band cut-offs, and
        // merges boundaries whose bands overlap into groups
        if (!grid_sync_last(ctl, a.flags, gen, lim, [&]() {
                resolve_cutoffs(ctl, Kb, N, d, s_keps, s_kabs, s_b, s_r, s_slot, s_sbin, s_nslot);
            }))
            return;
        const uint32_t K = __ldcg(&ctl->k_eff);       // boundaries of the epoch

        // ---- C: classify every point left: certainly in a round of the epoch, in a band, or later
        const uint32_t ng = __ldcg(&ctl->n_groups);
        if (t < (int)ng) {
            s_gin[t] = __ldcg(&ctl->g_in[t]);
            s_gout[t] = __ldcg(&ctl->g_out[t]);
            s_gq2[t] = __ldcg(&ctl->g_q2[t]);
        }
        if (t < kMaxEpoch) {
            s_cc[t] = 0;
            s_gc[t] = 0;
        }
        if (t == 0) s_glast = __ldcg(&ctl->g_out[ng - 1]);
        __syncthreads();
        classify_live(a, LV, n_live, Ls, r0, K, ng, s_gin, s_gout, s_gq2, s_glast, s_cc, s_gc);
        __syncthreads();
        if (t < (int)K && s_cc[t]) atomicAdd(&ctl->cert[t], s_cc[t]);
        if (t < (int)ng && s_gc[t]) atomicAdd(&ctl->gcnt[t], s_gc[t]);
        if (!grid_sync(ctl, a.flags, gen, lim)) return;

        // ---- D: the band entries regrouped by group with their compensated distances
        // (across the grid), then each group's band settled (CTA c takes groups c, c + G, ...)
        {
            const uint32_t nlist = __ldcg(&ctl->band_cnt);
            if (t < (int)ng) {
                uint32_t off = 0;
                for (uint32_t h = 0; h < (uint32_t)t; h++) off += __ldcg(&ctl->gcnt[h]);
                s_cc[t] = off;                       // the group's region in gkey / gpos
            }
            __syncthreads();
            // one slot claim per warp and group: the entries of a pass crowd into a few
            // groups, whose fill counters would otherwise take one contended atomic each
            for (uint32_t b0 = c * kThreads; b0 < nlist; b0 += G * kThreads) {     // warp-uniform bound
                const uint32_t e = b0 + (uint32_t)t;
                const bool v = e < nlist;
                const uint32_t k = v ? __ldcg(&a.band_k32[e]) : 0u;
                const uint32_t pos = v ? __ldcg(&a.band_pos[e]) : 0u;
                uint32_t g = 0;
                while (g + 1 < ng && k > s_gout[g]) g++;
                const uint32_t lane = (uint32_t)t & 31u;
                const uint32_t peers = __match_any_sync(0xffffffffu, v ? g : 0xFFFFFFFFu);
                const uint32_t leader = (uint32_t)__ffs(peers) - 1u;
                uint32_t slot = 0;
                if (v && lane == leader) slot = atomicAdd(&ctl->gfill[g], (uint32_t)__popc(peers));
                slot = __shfl_sync(0xffffffffu, slot, (int)leader) + (uint32_t)__popc(peers & ((1u << lane) - 1u));
                if (v) {
                    a.gkey[s_cc[g] + slot] = dff_key(a.x + (size_t)(pos & kPosMask) * d, Ls, d);
                    a.gpos[s_cc[g] + slot] = pos;
                }
            }
            if (!grid_sync(ctl, a.flags, gen, lim)) return;
            for (uint32_t g = c; g < ng; g += G) settle_group(a, Ls, g, r0, K, scr);
        }
        // the last CTA to arrive finds how many rounds the epoch commits: up to the first
        // round after which some attribute has no holder of its landmark value left
        if (!grid_sync_last(ctl, a.flags, gen, lim, [&]() { commit_count(a, Ls, K, r0, need_keys); }))
            return;

        // ---- E: commit: the epoch's first k_commit rounds leave the lists; the other
        // assignments are dropped; the next landmark if it changes
        uint32_t kcm = __ldcg(&ctl->k_commit);
        if (kcm < 1u || kcm > K) {                    // cannot happen; keeps the loop finite
            if (c == 0 && t == 0) atomicOr(&a.flags[1], 1u);
            kcm = 1u;
        }
        const bool changed = __ldcg(&ctl->l_changed) != 0;
        const uint32_t live_from = r0 + kcm;
        n_live = kc ? compact_shared(a, LV, n_live, r0, live_from, changed, scr)
                    : compact_global(a, LV, n_live, r0, live_from, changed, scr);
        if (!kc) {
            uint32_t *ti = gid; gid = gid2; gid2 = ti;
            uint32_t *tk = gkp; gkp = gkp2; gkp2 = tk;
            uint8_t *tf = gfl; gfl = gfl2; gfl2 = tf;
            pfl = gfl;
        }
        // the epoch's scratch, cleared across the grid for the next one
        {
            const uint32_t ns = __ldcg(&ctl->n_slots);
            uint32_t *h1 = &ctl->h1[0][0];
            for (uint32_t b = c * kThreads + t; b < ns * (uint32_t)kHistBins; b += G * kThreads) h1[b] = 0;
            uint32_t *hc = &ctl->hcnt[0][0];
            for (uint32_t b = c * kThreads + t; b < (uint32_t)d * kMaxEpoch; b += G * kThreads) hc[b] = 0;
            if (c == 0 && t < kMaxEpoch) {
                ctl->cert[t] = 0;
                ctl->bnd[t] = 0;
                ctl->gcnt[t] = 0;
                ctl->gfill[t] = 0;
            }
            if (c == 0 && t == 0) ctl->band_cnt = 0;
        }
        if (changed) find_landmark(a, lm_first, lm_step, live_from);
        first = false;
        need_keys = changed;
        r0 += kcm;
        if (!grid_sync(ctl, a.flags, gen, lim)) return;
    }
}

// ------------------------------------------------------------------ barrier cost
// The peel's grid barrier alone: `rounds` barriers in a row, in the peel's launch shape
// (the same block size, dynamic shared memory and CTAs per SM, so the same grid), timed
// to give the latency floor that the peel's barriers put under its epochs.
__global__ void __launch_bounds__(kThreads) k_barrier_bench(PeelCtl *ctl, uint32_t *flags, int rounds, unsigned lim)
{
    extern __shared__ __align__(16) uint32_t dyn[];
    if (threadIdx.x == 0 && rounds < 0) dyn[0] = 0;          // keeps the launch's shared memory
    unsigned gen = 0;
    for (int r = 0; r < rounds; r++)
        if (!grid_sync(ctl, flags, gen, lim)) return;
}

// ------------------------------------------------------------------ the points by attribute
// x (n x d, by point) into xt (d x n, by attribute) for the peel's key updates: 32 x 32
// tiles through shared memory, so that both the reads (32 attributes of a point) and the
// writes (32 points of an attribute) are coalesced.
constexpr int kTrThreads = 256;
constexpr size_t kTransposeBytes = size_t(96) << 20;

__global__ void __launch_bounds__(kTrThreads) k_transpose(const float *__restrict__ x, int64_t n, int d,
                                                          float *__restrict__ xt)
{
    __shared__ float tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t tiles_c = (d + 31) / 32;
    const int64_t tiles = (n + 31) / 32 * tiles_c;
    for (int64_t tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
        const int64_t r0 = tt / tiles_c * 32;
        const int c0 = (int)(tt % tiles_c) * 32;
        for (int k = ty; k < 32; k += kTrThreads / 32) {
            const int64_t r = r0 + k;
            if (r < n && c0 + tx < d) tile[k][tx] = __ldg(&x[r * d + c0 + tx]);
        }
        __syncthreads();
        for (int k = ty; k < 32; k += kTrThreads / 32) {
            const int64_t r = r0 + tx;
            if (r < n && c0 + k < d) xt[(size_t)(c0 + k) * (size_t)n + (size_t)r] = tile[tx][k];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ packing by round
// Stable counting sort of the points by round (8 bits of it per pass): the subclusters,
// each in ascending point index.  Chunk c of the items is [c m/G, (c+1) m/G).
constexpr int kPermThreads = 256;

__global__ void __launch_bounds__(kPermThreads) k_perm_count(const uint32_t *__restrict__ rnd,
                                                             const uint32_t *__restrict__ src, uint32_t m, int sh,
                                                             uint32_t *__restrict__ cnt)
{
    __shared__ uint32_t h[256];
    const int t = threadIdx.x;
    const uint32_t G = gridDim.x, c = blockIdx.x;
    h[t] = 0;
    __syncthreads();
    const uint32_t lo = (uint32_t)((uint64_t)c * m / G), hi = (uint32_t)((uint64_t)(c + 1) * m / G);
    for (uint32_t i = lo + t; i < hi; i += kPermThreads) {
        const uint32_t id = src ? __ldg(&src[i]) : i;
        atomicAdd(&h[(__ldg(&rnd[id]) >> sh) & 255u], 1u);
    }
    __syncthreads();
    cnt[(size_t)t * G + c] = h[t];
}

// Exclusive scan of the 256 x G counts in place (digit-major): one block of 1024 threads,
// each taking a run of consecutive counts (a multiple of 4, read and written as uint4 with
// several loads in flight: the scan is a chain of L2 round trips, not a bandwidth cost).
__global__ void __launch_bounds__(1024) k_perm_scan(uint32_t *cnt, uint32_t total)
{
    __shared__ uint32_t ws[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t per = (((total + 1023u) / 1024u) + 3u) & ~3u;        // total = 256 G, a multiple of 4
    const uint32_t b = min(total, (uint32_t)t * per), e = min(total, b + per);
    uint4 *c4 = reinterpret_cast<uint4 *>(cnt);
    uint32_t s = 0;
#pragma unroll 8
    for (uint32_t i = b; i < e; i += 4) {
        const uint4 v = c4[i / 4];
        s += v.x + v.y + v.z + v.w;
    }
    const uint32_t inc = warp_incl_scan(s);
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        const uint32_t v = ws[lane];
        ws[lane] = warp_incl_scan(v) - v;
    }
    __syncthreads();
    uint32_t run = ws[w] + inc - s;
#pragma unroll 8
    for (uint32_t i = b; i < e; i += 4) {
        const uint4 v = c4[i / 4];
        uint4 o;
        o.x = run;
        o.y = run + v.x;
        o.z = o.y + v.y;
        o.w = o.z + v.z;
        run = o.w + v.w;
        c4[i / 4] = o;
    }
}

__global__ void __launch_bounds__(kPermThreads) k_perm_scatter(const uint32_t *__restrict__ rnd,
                                                               const uint32_t *__restrict__ src, uint32_t m, int sh,
                                                               const uint32_t *__restrict__ cnt,
                                                               uint32_t *__restrict__ dst)
{
    constexpr int W = kPermThreads / 32;
    __shared__ uint32_t base[256];
    __shared__ uint32_t wc[W][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t G = gridDim.x, c = blockIdx.x;
    const uint32_t lt = (1u << lane) - 1u;
    base[t] = cnt[(size_t)t * G + c];
    const uint32_t lo = (uint32_t)((uint64_t)c * m / G), hi = (uint32_t)((uint64_t)(c + 1) * m / G);
    for (uint32_t i0 = lo; i0 < hi; i0 += kPermThreads) {
        const uint32_t i = i0 + t;
        const bool valid = i < hi;
        const uint32_t id = valid ? (src ? __ldg(&src[i]) : i) : 0u;
        const uint32_t dg = valid ? (__ldg(&rnd[id]) >> sh) & 255u : 256u;
        for (int q = t; q < W * 256; q += kPermThreads) (&wc[0][0])[q] = 0;
        __syncthreads();
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        if (valid && (peers & lt) == 0) wc[w][dg] = (uint32_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t o = base[dg] + (uint32_t)__popc(peers & lt);
            for (int v = 0; v < w; v++) o += wc[v][dg];
            dst[o] = id;
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int v = 0; v < W; v++) add += wc[v][t];
        base[t] += add;
        __syncthreads();
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
    // all control state starts cleared; the first landmark is the origin (the scaled
    // minimum of every attribute is exactly 0); no point has a round yet
    cudaError_t e = cudaMemsetAsync(b.ctl, 0, sizeof(PeelCtl), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b.bcnt, 0, (size_t)d * b.nbuckets * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b.rnd, 0xFF, (size_t)n * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b.pflag, kFlNone, (size_t)n, st);
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
    if (b.max_grid > 0 && grid > b.max_grid) grid = b.max_grid;
    PeelArgs a;
    a.x = b.x;
    // the points by attribute for the key updates, in xseg (idle until the subclusters are
    // gathered after the launch), where the rows do not fit in L2: an update then reads 4
    // bytes of each point left instead of a 32-byte sector of its row
    a.xt = (size_t)n * d * sizeof(float) > kTransposeBytes ? b.xseg : nullptr;
    a.d = d;
    a.n = n;
    a.N = N;
    a.S = S;
    a.rnd = b.rnd;
    a.pflag = b.pflag;
    a.ord = b.ord;
    a.bcnt = b.bcnt;
    a.bcs = b.bcs;
    a.lidx = b.lidx;
    a.kpos = b.kpos;
    a.ord_ld = b.ord_ld;
    a.nbk = b.nbuckets;
    a.band_k32 = b.band_k32;
    a.band_pos = b.band_pos;
    a.gkey = b.gkey;
    a.gpos = b.gpos;
    a.akey = b.akey;
    a.apos = b.apos;
    a.landmarks = b.landmarks;
    a.ctl = b.ctl;
    a.flags = b.flags;
    a.kmax = (uint32_t)(b.rounds_per_pass > 0 ? std::min(b.rounds_per_pass, kMaxEpoch) : kDefaultRounds);
    a.spin = b.wait_limit ? b.wait_limit : kDefaultSpin;
    a.stall = b.stall_first_barrier ? 1u : 0u;
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
    if (a.xt) {                  // timed and counted with the peel it serves
        k_transpose<<<sm_count * 8, kTrThreads, 0, st>>>(b.x, n, d, b.xseg);
        kt->launches[PSCL_K_PEEL]++;
    }
    e = cudaLaunchKernelEx(&cfg, k_peel<D>, a);
    kt->end(PSCL_K_PEEL, st);
    if (e != cudaSuccess) return e;
    // the subclusters packed by round: a stable counting sort, 8 bits of the round per pass
    int passes = 1;
    while (passes < 4 && (S - 1) >> (8 * passes)) passes++;
    const int pg = perm_grid(n, sm_count);
    const uint32_t m = (uint32_t)n;
    const uint32_t *src = nullptr;
    for (int p = 0; p < passes; p++) {
        uint32_t *dst = ((passes - 1 - p) & 1) ? b.gpos : b.perm;
        kt->begin(st);
        k_perm_count<<<pg, kPermThreads, 0, st>>>(b.rnd, src, m, 8 * p, b.pcnt);
        k_perm_scan<<<1, 1024, 0, st>>>(b.pcnt, (uint32_t)(256 * pg));
        k_perm_scatter<<<pg, kPermThreads, 0, st>>>(b.rnd, src, m, 8 * p, b.pcnt, dst);
        kt->end(PSCL_K_GATHER, st);
        src = dst;
    }
    e = cudaGetLastError();
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

cudaError_t measure_grid_barrier(int sm_count, double *us, bool *timed_out)
{
    const size_t smem = kPeelDynWords * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_barrier_bench, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // the peel's grid at full size: its CTAs per SM (capped at 4), as peel_launch sizes it
    e = cudaFuncSetAttribute(k_peel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel<16>, kThreads, smem);
    if (e != cudaSuccess) return e;
    int bench_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bench_sm, k_barrier_bench, kThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::min(std::min(per_sm, 4), bench_sm);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::min(sm_count * per_sm, kMaxPeelGrid);
    PeelCtl *ctl = nullptr;
    uint32_t *flags = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    constexpr int kRounds = 2000;
    float best = 0.0f;
    uint32_t hf[2] = {0u, 0u};
    if ((e = cudaMalloc(&ctl, sizeof(PeelCtl))) == cudaSuccess && (e = cudaMalloc(&flags, 8)) == cudaSuccess &&
        (e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) == cudaSuccess &&
        (e = cudaEventCreate(&t0)) == cudaSuccess && (e = cudaEventCreate(&t1)) == cudaSuccess) {
        for (int r = 0; r < 4 && e == cudaSuccess; r++) {        // the first a warm-up
            cudaMemsetAsync(ctl, 0, sizeof(PeelCtl), st);
            cudaMemsetAsync(flags, 0, 8, st);
            int rounds = kRounds;
            unsigned lim = kDefaultSpin;
            void *args[] = {&ctl, &flags, &rounds, &lim};
            cudaEventRecord(t0, st);
            e = cudaLaunchCooperativeKernel((const void *)k_barrier_bench, dim3(grid), dim3(kThreads), args, smem, st);
            cudaEventRecord(t1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            if (e == cudaSuccess) e = cudaMemcpy(hf, flags, 8, cudaMemcpyDeviceToHost);
            float ms = 0.0f;
            if (e == cudaSuccess) cudaEventElapsedTime(&ms, t0, t1);
            if (r > 0 && (best == 0.0f || ms < best)) best = ms;
            if (hf[1]) break;
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (st) cudaStreamDestroy(st);
    cudaFree(flags);
    cudaFree(ctl);
    if (e != cudaSuccess) return e;
    *timed_out = hf[1] != 0u;
    *us = 1e3 * (double)best / kRounds;
    return cudaSuccess;
}

uint32_t peel_buckets(int64_t n)
{
    uint32_t nb = 4096;
    while (nb < 65536u && (int64_t)nb * 16 < n) nb <<= 1;
    return nb;
}

int perm_grid(int64_t n, int sm_count)
{
    int64_t g = (n + 2047) / 2048;
    if (g > (int64_t)sm_count * 4) g = (int64_t)sm_count * 4;
    return (int)std::max<int64_t>(1, g);
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
