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
//   A. delta32_i by a float32 FMA chain, kept as its bit pattern (order-preserving for
//      non-negative floats), and a 2048-bin histogram of key bits 31..21;
//   B. the bin holding the N-th smallest key, and a 2048-bin histogram of bits 20..10 of
//      the keys inside it: the N-th smallest key lies in a 22-bit prefix [A, B];
//   C. |delta32 - delta64| <= eps*delta32 + ea with eps = (d+4)*2^-23, ea = 2^-120, so
//      the N-th smallest delta64 lies in [A(1-eps)-ea, B(1+eps)+ea]: a point whose upper
//      bound is below that interval is certainly taken, one whose lower bound is above
//      it certainly not; the few in between (the band) get delta64 exactly as defined;
//   D. the (N - #certain) smallest band points by (delta64, position) are taken; taken
//      points go to subcluster r in ascending index, the rest stay in ascending index
//      (stable compaction of indices), and the per-attribute minimum of the points that
//      stay is the next landmark.
// The partition is therefore exactly the float64 definition's, whatever float32 does.
//
// All rounds run in one persistent cooperative launch: every CTA owns a contiguous slice
// of the remaining points in each round and the phases are separated by grid barriers
// (four per round).  Every barrier wait is bounded; a CTA that gives up sets the abort
// flag, every other CTA then leaves at its next wait, and the host sees PSCL_ETIMEOUT.
#include <algorithm>

#include "pscl_internal.cuh"

namespace pscl {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kInfBits = 0x7f800000u;
constexpr int kBandSmem = 1024;               // band entries settled in shared memory
constexpr int kBandBins = 4096;               // one-ulp bins over a band's float32 keys
constexpr int kTight = 256;                   // band entries near the cut-off, decided exactly
constexpr int kPeelDynWords = 2 * kHistBins > kBandBins + 7 * kTight
                                  ? 2 * kHistBins : kBandBins + 7 * kTight;
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

// ------------------------------------------------------------------ the kernel
struct PeelArgs {
    const float *x;
    int d;
    int64_t n, N, S;
    uint32_t *idx0, *idx1;       // remaining indices, ping-pong
    uint32_t *key;
    uint8_t *status;             // 0 out, 1 taken, 2 band
    uint64_t *band_key;          // float64 distance bits (wide bands only)
    uint32_t *band_k32;          // float32 keys of the band
    uint32_t *band_pos;
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

template <int D>
__global__ void __launch_bounds__(kThreads) k_peel(PeelArgs a)
{
    constexpr int DM = D > 0 && D <= 64 ? D : 1;       // register minima when D is small
    constexpr int B = kPeelBatch<D>();
    constexpr int QT = 16;                             // tiles of kThreads items per scan
    constexpr int W = kThreads / 32;
    // dynamic shared memory: [first histogram | guessed second-digit histogram], all of
    // it reused for the band in phase D
    extern __shared__ __align__(16) uint32_t dyn[];
    uint32_t *sh = dyn;
    uint32_t *gh = dyn + kHistBins;
    __shared__ float Ls[D > 0 ? D : kMaxD];
    __shared__ uint32_t s_in_key, s_out_key, s_nt, s_na, s_v, s_t32;
    __shared__ float wmin[W][DM];
    __shared__ uint32_t gmin[D > 0 && D <= 64 ? 1 : kMaxD];
    __shared__ uint32_t off_t[QT * W], off_u[QT * W], s_tot[2];
    PeelCtl *ctl = a.ctl;
    const int d = a.d;
    const int t = threadIdx.x;
    const int lane = t & 31, w = t >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const unsigned G = gridDim.x, c = blockIdx.x;
    unsigned gen = 0;
    uint32_t guess = 0xFFFFFFFFu;      // first digit of the previous round's N-th key

    for (int64_t r = 0; r < a.S; r++) {
        const int64_t nr = a.n - r * a.N;
        const int par = (int)(r & 1);
        const uint32_t *idx_in = r == 0 ? nullptr : (par ? a.idx1 : a.idx0);
        uint32_t *idx_out = par ? a.idx0 : a.idx1;
        uint32_t *seg_out = a.perm + r * a.N;
        const uint32_t s0 = (uint32_t)((int64_t)c * nr / G), s1 = (uint32_t)((int64_t)(c + 1) * nr / G);
        if (nr <= a.N) {                              // the last subcluster: all that is left
            for (uint32_t i = s0 + t; i < s1; i += kThreads) seg_out[i] = idx_in ? __ldcg(&idx_in[i]) : i;
            if (c == 0 && a.landmarks)
                for (int j = t; j < d; j += kThreads)
                    a.landmarks[r * d + j] = __uint_as_float(__ldcg(&ctl->Lbits[par][j]));
            break;
        }
        uint32_t *hist0 = ctl->hist[par][0], *hist1 = ctl->hist[par][1];

        // ---- A: float32 distances and the first histogram
        for (int j = t; j < d; j += kThreads) Ls[j] = __uint_as_float(__ldcg(&ctl->Lbits[par][j]));
        const bool have_guess = guess != 0xFFFFFFFFu;
        for (int b = t; b < (have_guess ? 2 : 1) * kHistBins; b += kThreads) dyn[b] = 0;
        if (c == 0) {
            for (int j = t; j < d; j += kThreads) {
                ctl->Lbits[par ^ 1][j] = kInfBits;
                if (a.landmarks) a.landmarks[r * d + j] = __uint_as_float(__ldcg(&ctl->Lbits[par][j]));
            }
            if (t == 0) ctl->band_cnt[par ^ 1] = 0;
        }
        __syncthreads();
        for (uint32_t i0 = s0 + t; i0 < s1; i0 += B * kThreads) {
            uint32_t rows[B];
#pragma unroll
            for (int q = 0; q < B; q++) {
                const uint32_t i = i0 + q * kThreads;
                rows[q] = i < s1 ? (idx_in ? __ldcg(&idx_in[i]) : i) : 0u;
            }
            float dl[B];
#pragma unroll
            for (int q = 0; q < B; q++) dl[q] = dist32<D>(a.x + (size_t)rows[q] * d, Ls, d);
#pragma unroll
            for (int q = 0; q < B; q++) {
                const uint32_t i = i0 + q * kThreads;
                if (i < s1) {
                    const uint32_t k = __float_as_uint(dl[q]);
                    a.key[i] = k;
                    atomicAdd(&sh[k >> 21], 1u);
                    if (have_guess && (k >> 21) == guess) atomicAdd(&gh[(k >> 10) & (kHistBins - 1)], 1u);
                }
            }
        }
        __syncthreads();
        for (int b = t; b < kHistBins; b += kThreads)
            if (sh[b]) atomicAdd(&hist0[b], sh[b]);
        if (have_guess) {
            uint32_t *gg = &ctl->ghist[par][0];
            for (int b = t; b < kHistBins; b += kThreads)
                if (gh[b]) atomicAdd(&gg[b], gh[b]);
        }
        if (!grid_sync(ctl, a.flags, gen)) return;

        // ---- B: second histogram inside the N-th key's bin (skipped when the bin was
        // guessed: the previous round's N-th key is almost always in the same bin)
        uint32_t b0, rank0;
        find_bin(hist0, (uint32_t)(a.N - 1), b0, rank0);
        const bool hit = have_guess && b0 == guess;
        guess = b0;
        if (hit) {
            hist1 = &ctl->ghist[par][0];
        } else {
        for (int b = t; b < kHistBins; b += kThreads) sh[b] = 0;
        __syncthreads();
        for (uint32_t i0 = s0 + t; i0 < s1; i0 += 4 * kThreads) {
            uint32_t k4[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t i = i0 + q * kThreads;
                k4[q] = i < s1 ? a.key[i] : 0xFFFFFFFFu;
            }
#pragma unroll
            for (int q = 0; q < 4; q++)
                if ((k4[q] >> 21) == b0 && k4[q] != 0xFFFFFFFFu) atomicAdd(&sh[(k4[q] >> 10) & (kHistBins - 1)], 1u);
        }
        __syncthreads();
        for (int b = t; b < kHistBins; b += kThreads)
            if (sh[b]) atomicAdd(&hist1[b], sh[b]);
        if (!grid_sync(ctl, a.flags, gen)) return;
        }

        // ---- C: classify; the band is listed
        uint32_t b1, rank1;
        find_bin(hist1, rank0, b1, rank1);
        if (t == 0) band_cutoffs(b0, b1, d, s_in_key, s_out_key);
        {   // clear next round's histograms (last read in the previous round)
            uint32_t *nh = &ctl->hist[par ^ 1][0][0];
            for (uint32_t b = c * kThreads + t; b < 2u * kHistBins; b += G * kThreads) nh[b] = 0;
            uint32_t *ng = &ctl->ghist[par ^ 1][0];
            for (uint32_t b = c * kThreads + t; b < (uint32_t)kHistBins; b += G * kThreads) ng[b] = 0;
        }
        __syncthreads();
        const uint32_t in_key = s_in_key, out_key = s_out_key;
        uint32_t n_in = 0;
        for (uint32_t i0 = s0 + t; i0 < s1; i0 += 4 * kThreads) {
            uint32_t k4[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t i = i0 + q * kThreads;
                k4[q] = i < s1 ? a.key[i] : 0u;
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t i = i0 + q * kThreads;
                if (i >= s1) continue;
                const uint32_t k = k4[q];
                uint8_t s = k < in_key ? 1 : (k > out_key ? 0 : 2);
                if (s == 2) {
                    const uint32_t slot = atomicAdd(&ctl->band_cnt[par], 1u);
                    a.band_k32[slot] = k;
                    a.band_pos[slot] = i;
                }
                n_in += s == 1;
                a.status[i] = s;
            }
        }
        n_in = block_sum(n_in);
        if (t == 0) ctl->cnt_in[c] = n_in;
        if (!grid_sync(ctl, a.flags, gen)) return;

        // ---- D: settle the band, compact, next landmark
        uint32_t all_in = 0, in_before = 0;
        for (uint32_t q = t; q < G; q += kThreads) {
            const uint32_t v = __ldcg(&ctl->cnt_in[q]);
            all_in += v;
            if (q < c) in_before += v;
        }
        all_in = block_sum(all_in);
        in_before = block_sum(in_before);
        const uint32_t nb = __ldcg(&ctl->band_cnt[par]);
        const uint32_t need = (uint32_t)a.N > all_in ? (uint32_t)a.N - all_in : 0u;
        if ((all_in > (uint32_t)a.N || need > nb) && c == 0 && t == 0) atomicOr(&a.flags[1], 1u);
        uint32_t band_before = 0;
        bool slow = false;
        if (need > 0 && need < nb) {
            // Fast path, in shared memory (every CTA redundantly).  The need-th smallest
            // float32 key T32 of the band comes from a one-ulp histogram; the float32 error
            // bound around T32 leaves a tight set of a few entries; their distances in
            // compensated float32 (dff, within eps_ff of the float64 definition) settle all
            // of them but those within the dff error of the cut-off (in practice only exact
            // ties), which are decided in float64.
            uint32_t *hb = dyn;                                    // kBandBins one-ulp bins
            uint32_t *tpos = dyn + kBandBins;                      // kTight tight entries
            float *th = reinterpret_cast<float *>(tpos + kTight);
            float *tl = th + kTight;
            uint32_t *tcls = reinterpret_cast<uint32_t *>(tl + kTight);   // 1 taken, 0 not
            uint32_t *tamb = tcls + kTight;                        // undecided tight entries
            unsigned long long *td = reinterpret_cast<unsigned long long *>(tamb + kTight);
            const uint32_t range = out_key - in_key + 1u;
            slow = range > (uint32_t)kBandBins;
            if (!slow) {
                for (int b = t; b < kBandBins; b += kThreads) hb[b] = 0;
                if (t == 0) {
                    s_nt = 0;
                    s_na = 0;
                }
                __syncthreads();
                for (uint32_t q = t; q < nb; q += kThreads) atomicAdd(&hb[__ldcg(&a.band_k32[q]) - in_key], 1u);
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
                uint32_t tin, tout;
                band_cutoffs_key(s_t32, s_t32, d, tin, tout);
                uint32_t n_cert = 0;
                for (uint32_t q = t; q < nb; q += kThreads) {
                    const uint32_t k = __ldcg(&a.band_k32[q]);
                    if (k < tin) {
                        n_cert++;
                    } else if (k <= tout) {
                        const uint32_t slot = atomicAdd(&s_nt, 1u);
                        if (slot < (uint32_t)kTight) tpos[slot] = __ldcg(&a.band_pos[q]);
                    }
                }
                n_cert = block_sum(n_cert);
                const uint32_t nt = s_nt;
                slow = nt > (uint32_t)kTight || n_cert > need || need - n_cert > nt;
                if (!slow) {
                    const uint32_t need2 = need - n_cert;
                    for (uint32_t q = t; q < nt; q += kThreads) {
                        const uint32_t pq = tpos[q];
                        const uint32_t row = idx_in ? __ldcg(&idx_in[pq]) : pq;
                        float h, l;
                        dist_ff(a.x + (size_t)row * d, Ls, d, h, l);
                        th[q] = h;
                        tl[q] = l;
                    }
                    __syncthreads();
                    // V: the tight entry of rank need2-1 in (dff, position) order
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
                        uint32_t cls = diff < -win ? 1u : 0u;
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
                        for (uint32_t q = t; q < na; q += kThreads) {
                            const uint32_t pq = tpos[tamb[q]];
                            const uint32_t row = idx_in ? __ldcg(&idx_in[pq]) : pq;
                            td[q] = (unsigned long long)__double_as_longlong(dist64(a.x + (size_t)row * d, Ls, d));
                        }
                        __syncthreads();
                        for (uint32_t q = t; q < na; q += kThreads) {
                            const unsigned long long kq = td[q];
                            const uint32_t pq = tpos[tamb[q]];
                            uint32_t rk = 0;
                            for (uint32_t o = 0; o < na; o++) rk += (td[o] < kq) || (td[o] == kq && tpos[tamb[o]] < pq);
                            tcls[tamb[q]] = rk < need3 ? 1u : 0u;
                        }
                    }
                    __syncthreads();
                    for (uint32_t q = t; q < nb; q += kThreads) {
                        const uint32_t k = __ldcg(&a.band_k32[q]);
                        const uint32_t pq = __ldcg(&a.band_pos[q]);
                        bool take = k < tin;
                        if (!take && k <= tout)
                            for (uint32_t o = 0; o < nt; o++)
                                if (tpos[o] == pq) take = tcls[o] != 0;
                        if (take) {
                            if (pq < s0) band_before++;
                            else if (pq < s1) a.status[pq] = 1;
                        }
                    }
                }
                __syncthreads();
            }
            if (slow) {
                // wide band (e.g. many equal distances): float64 for every band entry, spread
                // over all CTAs, then one CTA selects while the rest wait
                for (uint32_t q = c * kThreads + t; q < nb; q += G * kThreads) {
                    const uint32_t pq = __ldcg(&a.band_pos[q]);
                    const uint32_t row = idx_in ? __ldcg(&idx_in[pq]) : pq;
                    a.band_key[q] = (uint64_t)__double_as_longlong(dist64(a.x + (size_t)row * d, Ls, d));
                }
                if (!grid_sync(ctl, a.flags, gen)) return;
                uint64_t K = 0;
                uint32_t Pp = 0;
                if (c == 0) {
                    select_band_global(a.band_key, a.band_pos, nb, need, K, Pp);
                    if (t == 0) {
                        ctl->sel_key = K;
                        ctl->sel_pos = Pp;
                    }
                }
                if (!grid_sync(ctl, a.flags, gen)) return;
                K = __ldcg(&ctl->sel_key);
                Pp = __ldcg(&ctl->sel_pos);
                band_before = 0;
                for (uint32_t q = t; q < nb; q += kThreads) {
                    const uint64_t kq = __ldcg(&a.band_key[q]);
                    const uint32_t pq = __ldcg(&a.band_pos[q]);
                    if (kq < K || (kq == K && pq <= Pp)) {
                        if (pq < s0) band_before++;
                        else if (pq < s1) a.status[pq] = 1;
                    }
                }
            }
        } else if (need > 0) {
            // need >= nb: the whole band is taken (need > nb contradicts the bound; flagged)
            for (uint32_t q = t; q < nb; q += kThreads) {
                const uint32_t pq = __ldcg(&a.band_pos[q]);
                if (pq < s0) band_before++;
                else if (pq < s1) a.status[pq] = 1;
            }
        }
        band_before = block_sum(band_before);       // its barrier also orders the status writes
        uint32_t sel_base = in_before + band_before;
        uint32_t uns_base = s0 - sel_base;

        float mn[DM];
#pragma unroll
        for (int j = 0; j < DM; j++) mn[j] = __int_as_float(kInfBits);
        if (!(D > 0 && D <= 64)) {
            for (int j = t; j < d; j += kThreads) gmin[j] = kInfBits;
            __syncthreads();
        }
        // stable compaction, QT tiles of kThreads items per scan: item (q, t) of a chunk
        // is preceded by the earlier tiles, by the earlier warps of its tile and by the
        // lower lanes of its warp
        for (uint32_t cb = s0; cb < s1; cb += QT * kThreads) {
            uint32_t tk = 0, vl = 0;                 // bit q: item (q, t) taken / valid
            uint32_t ids[QT];
#pragma unroll
            for (int q = 0; q < QT; q++) {
                const uint32_t i = cb + q * kThreads + t;
                const bool v = i < s1;
                const uint8_t st = v ? a.status[i] : 0;
                ids[q] = v ? (idx_in ? __ldcg(&idx_in[i]) : i) : 0u;
                vl |= (uint32_t)v << q;
                tk |= (uint32_t)(st == 1) << q;
            }
#pragma unroll
            for (int q = 0; q < QT; q++) {
                const uint32_t bt = __ballot_sync(0xffffffffu, (tk >> q) & 1u);
                const uint32_t bv = __ballot_sync(0xffffffffu, (vl >> q) & 1u);
                if (lane == 0) {
                    off_t[q * W + w] = __popc(bt);
                    off_u[q * W + w] = __popc(bv & ~bt);
                }
            }
            __syncthreads();
            if (w == 0) {                           // exclusive scan of the QT*W counts in order
                constexpr int PER = QT * W / 32;
                uint32_t at[PER], au[PER], st_ = 0, su = 0;
#pragma unroll
                for (int e = 0; e < PER; e++) {
                    at[e] = off_t[lane * PER + e];
                    au[e] = off_u[lane * PER + e];
                    st_ += at[e];
                    su += au[e];
                }
                uint32_t it = warp_incl_scan(st_), iu = warp_incl_scan(su);
                uint32_t et = it - st_, eu = iu - su;
#pragma unroll
                for (int e = 0; e < PER; e++) {
                    off_t[lane * PER + e] = et;
                    off_u[lane * PER + e] = eu;
                    et += at[e];
                    eu += au[e];
                }
                if (lane == 31) {
                    s_tot[0] = it;
                    s_tot[1] = iu;
                }
            }
            __syncthreads();
            uint32_t urows[QT];
            int nu = 0;
#pragma unroll
            for (int q = 0; q < QT; q++) {
                const uint32_t bt = __ballot_sync(0xffffffffu, (tk >> q) & 1u);
                const uint32_t bv = __ballot_sync(0xffffffffu, (vl >> q) & 1u);
                if ((vl >> q) & 1u) {
                    if ((tk >> q) & 1u) {
                        seg_out[sel_base + off_t[q * W + w] + __popc(bt & lt_mask)] = ids[q];
                    } else {
                        idx_out[uns_base + off_u[q * W + w] + __popc(bv & ~bt & lt_mask)] = ids[q];
                        urows[nu++] = ids[q];
                    }
                }
            }
            // minima of the rows that stay, B rows in flight at a time
            if (D > 0 && D <= 64) {
                for (int q0 = 0; q0 < nu; q0 += B) {
                    float rv[B][DM];
#pragma unroll
                    for (int q = 0; q < B; q++) {
                        const uint32_t id = q0 + q < nu ? urows[q0 + q] : urows[q0];
                        const float *row = a.x + (size_t)id * d;
                        if (DM % 4 == 0) {
                            const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
                            for (int j4 = 0; j4 < DM / 4; j4++) {
                                const float4 v = __ldg(&r4[j4]);
                                rv[q][4 * j4 + 0] = v.x;
                                rv[q][4 * j4 + 1] = v.y;
                                rv[q][4 * j4 + 2] = v.z;
                                rv[q][4 * j4 + 3] = v.w;
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < DM; j++) rv[q][j] = __ldg(&row[j]);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < B; q++)
#pragma unroll
                        for (int j = 0; j < DM; j++) mn[j] = fminf(mn[j], rv[q][j]);
                }
            } else {
                for (int q = 0; q < nu; q++) {
                    const float *row = a.x + (size_t)urows[q] * d;
                    for (int j = 0; j < d; j++) atomicMin(&gmin[j], __float_as_uint(__ldg(&row[j])));
                }
            }
            sel_base += s_tot[0];
            uns_base += s_tot[1];
            __syncthreads();
        }
        if (D > 0 && D <= 64) {
#pragma unroll
            for (int j = 0; j < DM; j++) {
                float v = mn[j];
                for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
                if (lane == 0) wmin[w][j] = v;
            }
            __syncthreads();
            for (int j = t; j < d; j += kThreads) {
                float v = wmin[0][j];
                for (int q = 1; q < W; q++) v = fminf(v, wmin[q][j]);
                if (__float_as_uint(v) < kInfBits) atomicMin(&ctl->Lbits[par ^ 1][j], __float_as_uint(v));
            }
        } else {
            __syncthreads();
            for (int j = t; j < d; j += kThreads)
                if (gmin[j] < kInfBits) atomicMin(&ctl->Lbits[par ^ 1][j], gmin[j]);
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
    const size_t smem = kPeelDynWords * sizeof(uint32_t);
    e = cudaFuncSetAttribute(k_peel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel<D>, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)sm_count * std::min(per_sm, 4);
    if (grid > kMaxPeelGrid) grid = kMaxPeelGrid;
    const int64_t want = (n + 63) / 64;             // at least ~64 points per CTA in round 0
    if (grid > want) grid = std::max<int64_t>(1, want);
    PeelArgs a;
    a.x = b.x;
    a.d = d;
    a.n = n;
    a.N = N;
    a.S = S;
    a.idx0 = b.idx[0];
    a.idx1 = b.idx[1];
    a.key = b.key;
    a.status = b.status;
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
    case 2: return peel_launch<2>(b, n, d, N, sm_count, st, kt);
    case 4: return peel_launch<4>(b, n, d, N, sm_count, st, kt);
    case 8: return peel_launch<8>(b, n, d, N, sm_count, st, kt);
    case 16: return peel_launch<16>(b, n, d, N, sm_count, st, kt);
    case 32: return peel_launch<32>(b, n, d, N, sm_count, st, kt);
    case 64: return peel_launch<64>(b, n, d, N, sm_count, st, kt);
    default: return peel_launch<0>(b, n, d, N, sm_count, st, kt);
    }
}

}  // namespace pscl
