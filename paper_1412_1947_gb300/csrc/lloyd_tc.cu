// Lloyd assignment step on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// For a tile of 128 rows x and the k centers c of their set, with every coordinate
// centred on a per-set reference point r (x~ = x - r, c~ = c - r; distances unchanged),
//     v_j = ||c~_j||^2 - 2 x~ . c~_j        (= ||x - c_j||^2 - ||x~||^2)
// is one MMA over K: A = [x~ terms, 1 ...] (128 x K), B = [-2 c~ terms, n parts] (k x K),
// with n parts summing to ||c~_j||^2 (split so that they survive the operand rounding).
// Modes (pscl_prec):
//   TF32    A = [x~], B = [-2c~]                     (one product per attribute)
//   BF16    likewise with BF16 operands
//   TF32X3  x~ = h + l, c~ = H + L split into TF32 parts: A = [h, h, l], B = [-2H, -2L, -2H]
//           so one MMA sums h.H + h.L + l.H (error ~2^-21 per product instead of ~2^-10)
//   BF16X3  likewise with BF16 parts (error ~2^-17 per product)
// The accumulator is float32 in tensor memory.  Each of the 128 threads owns one row (one
// TMEM lane), reads its k accumulators with tcgen05.ld and keeps the best and second best.
//
// Near ties: |v_j - exact| <= E = alpha ||x~|| cmax + beta cmax^2 (operand rounding,
// float32 accumulation over K terms, centring and norm errors; cmax = max_j ||c~_j||), plus
// the float32 error of a direct distance.  Every center within 2E of the best is re-scored
// with the float32 direct sum (x_i - c_ji)^2 -- the PSCL_PREC_FP32 arithmetic -- and the
// smallest, lowest index on ties, wins.  No center outside that set can win the float32
// direct comparison, so the labels equal those of the float32 direct path in every mode.
//
// Operands are written to shared memory by the threads in the canonical K-major layout
// without swizzle (8-row x 16-byte core matrices; the K-adjacent ones of a row group are
// contiguous, LBO = 128 bytes; row groups are SBO = K * element bytes apart).  Tiles are
// pipelined two deep: the operands and MMA of tile i+1 are issued before the epilogue of
// tile i (two operand buffers, two TMEM regions, two mbarriers).  One thread issues the
// MMAs and commits them to an mbarrier that every thread waits on with a bounded spin.
// The centroid sums are the same exact fixed-point sums as in the float32 path.
#include <cuda_bf16.h>

#include <algorithm>

#include "pscl_internal.cuh"

namespace pscl {
namespace {

constexpr int kTcThreads = 128;           // one thread per TMEM lane / tile row
constexpr int kTileRows = 128;            // MMA M
constexpr unsigned kWaitLimit = 1u << 26; // bounded mbarrier polls
constexpr float kFix = 4294967296.0f;
constexpr size_t kTcSmemMax = 200 * 1024; // dynamic shared memory the kernel may use

enum TcMode { kModeTf32 = 0, kModeBf16 = 1, kModeTf32x3 = 2, kModeBf16x3 = 3 };

__device__ __forceinline__ unsigned long long to_fix(float v)
{
    return (unsigned long long)__float2ll_rn(v * kFix);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ float bf16_rn(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <int MODE>
struct Op {
    static constexpr bool kBf16 = MODE == kModeBf16 || MODE == kModeBf16x3;
    static constexpr int kTerms = MODE >= kModeTf32x3 ? 3 : 1;    // operand blocks of D
    static constexpr int kBytes = kBf16 ? 2 : 4;
    static constexpr int kPerChunk = 16 / kBytes;
    static constexpr int kMmaK = kBf16 ? 16 : 8;
    static constexpr int kNormParts = kBf16 ? 3 : 2;
    // operand rounding to this mode's type
    static __device__ __forceinline__ float rnd(float x) { return kBf16 ? bf16_rn(x) : tf32_rna(x); }
    // relative error of one product of the rounded / split operands
    static __device__ __forceinline__ float eta_p()
    {
        switch (MODE) {
        case kModeTf32: return 0x1p-10f;
        case kModeBf16: return 0x1p-8f;
        case kModeTf32x3: return 3.0f * 0x1p-22f;
        default: return 3.0f * 0x1p-18f;
        }
    }
    // instruction descriptor: D f32, A/B tf32 (2) or bf16 (1), both K-major, N, M = 128
    static __device__ __forceinline__ uint32_t idesc(int n)
    {
        const uint32_t f = kBf16 ? 1u : 2u;
        return (1u << 4) | (f << 7) | (f << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTileRows >> 4) << 24);
    }
};

template <int D, int MODE>
struct TcLayout {
    using O = Op<MODE>;
    static constexpr int kUsed = O::kTerms * D + O::kNormParts;
    static constexpr int kK = ((kUsed + O::kMmaK - 1) / O::kMmaK) * O::kMmaK;
    static constexpr int kChunks = kK / O::kPerChunk;
    static constexpr uint32_t kGroup = kChunks * 128;                    // bytes per 8-row group
    static constexpr uint32_t kABytes = (kTileRows / 8) * kGroup;
};

// Element e of an A row from the split parts of x~ (h, l) of this row.
template <int D, int MODE>
__device__ __forceinline__ float a_elem(int e, const float *h, const float *l, bool live)
{
    using O = Op<MODE>;
    if (e < D) return h[e];
    if (O::kTerms == 3) {
        if (e < 2 * D) return h[e - D];
        if (e < 3 * D) return l[e - 2 * D];
    }
    if (e < O::kTerms * D + O::kNormParts) return live ? 1.0f : 0.0f;
    return 0.0f;
}

// Write one row of an operand (K elements from `elem`) as 16-byte chunks.
template <int D, int MODE, class F>
__device__ __forceinline__ void put_row(unsigned char *base, int row, F elem)
{
    using O = Op<MODE>;
    using L = TcLayout<D, MODE>;
    unsigned char *rp = base + (size_t)(row >> 3) * L::kGroup + (row & 7) * 16;
#pragma unroll
    for (int c = 0; c < L::kChunks; c++) {
        uint4 w;
        if (O::kBf16) {
            uint32_t v[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const __nv_bfloat16 lo = __float2bfloat16_rn(elem(c * 8 + 2 * q));
                const __nv_bfloat16 hi = __float2bfloat16_rn(elem(c * 8 + 2 * q + 1));
                v[q] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
            }
            w = make_uint4(v[0], v[1], v[2], v[3]);
        } else {
            w = make_uint4(__float_as_uint(elem(c * 4 + 0)), __float_as_uint(elem(c * 4 + 1)),
                           __float_as_uint(elem(c * 4 + 2)), __float_as_uint(elem(c * 4 + 3)));
        }
        *reinterpret_cast<uint4 *>(rp + c * 128) = w;
    }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; q++) v[q] = __uint_as_float(r[q]);
}

// Bounded wait for the mbarrier phase `parity`; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (unsigned it = 0; it < kWaitLimit; it++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// One thread: the K/kMmaK MMAs of a 128-row tile (A at a_smem, B at b_smem, D at TMEM
// column dcol), then a commit that arrives on the mbarrier at mbar_smem when they finish.
template <int D, int MODE>
__device__ __forceinline__ void issue_mma(uint32_t dcol, uint32_t a_smem, uint32_t b_smem, uint32_t idesc,
                                          uint32_t mbar_smem)
{
    using L = TcLayout<D, MODE>;
    using O = Op<MODE>;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int kb = 0; kb < L::kK / O::kMmaK; kb++) {
        const uint64_t ad = smem_desc(a_smem + 2 * kb * 128, 128, L::kGroup);
        const uint64_t bd = smem_desc(b_smem + 2 * kb * 128, 128, L::kGroup);
        const uint32_t accum = kb > 0;
        if (O::kBf16) {
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                         ::"r"(dcol), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
        } else {
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                         ::"r"(dcol), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_smem));
}

__device__ __host__ __forceinline__ uint32_t tmem_cols(int np)
{
    return np <= 32 ? 32u : (np <= 64 ? 64u : (np <= 128 ? 128u : 256u));
}

// The sums of a run are kept as two 32-bit halves of the 32.32 fixed-point value, q >> 16
// (<= 2^16 for coordinates in [0, 1]) and q & 0xFFFF, so 32768 rows can be added before
// either half could wrap; they are folded into the 64-bit global sums that often.
constexpr int kFoldTiles = 32768 / kTileRows;

__device__ __forceinline__ void flush_sums(uint32_t *shi, uint32_t *slo, int32_t *scnt, int k, int64_t c0,
                                           unsigned long long *acc, int32_t *count, int dd)
{
    const int ds = dd | 1;
    for (int e = threadIdx.x; e < k * dd; e += kTcThreads) {
        const int c = e / dd, es = c * ds + (e - c * dd);
        const unsigned long long v = ((unsigned long long)shi[es] << 16) + slo[es];
        if (v) atomicAdd(&acc[c0 * dd + e], v);
        shi[es] = 0u;
        slo[es] = 0u;
    }
    for (int j = threadIdx.x; j < k; j += kTcThreads) {
        const int v = scnt[j];
        if (v) atomicAdd(&count[c0 + j], v);
        scnt[j] = 0;
    }
}

// One assignment step.  CTA c serves the units [split[c], split[c+1]) (a persistent
// launch over all units) or the single unit unit_lo + c (split == NULL).  Its units form
// runs of consecutive units of one set; per run the set's operand B, reference point and
// sums are set up once and its rows stream through the tensor cores in 128-row tiles,
// two deep when two TMEM regions of ncols columns fit (nbuf = 2), else one at a time.
template <int D, int MODE>
__global__ void __launch_bounds__(kTcThreads)
k_lloyd_assign_tc(const float *__restrict__ pts, SegTable t, const int32_t *split, int unit_lo,
                  const float *__restrict__ centers, unsigned long long *acc, int32_t *count, int32_t *labels,
                  int32_t *trace, int64_t trace_off, int kmax, int nbuf, uint32_t ncols, int sacc, int scent,
                  uint32_t *flags)
{
    using L = TcLayout<D, MODE>;
    using O = Op<MODE>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ float s_ref[D];
    __shared__ float s_part[kTcThreads];
    __shared__ float s_cmax2;
    __shared__ int s_fail;
    __shared__ uint32_t s_stat[2];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ub = split ? split[blockIdx.x] : unit_lo + (int)blockIdx.x;
    const int ue = split ? split[blockIdx.x + 1] : ub + 1;
    const int npmax = (kmax + 15) & ~15;

    // [A buffers | B | float32 centers (scent) | high sums | low sums | counts (sacc)]; a
    // center's sums take the odd stride D | 1 so that a warp's lanes adding one attribute
    // of different centers spread over the banks
    constexpr int DS = D | 1;
    unsigned char *sa0 = smem;
    unsigned char *sb = sa0 + (size_t)nbuf * L::kABytes;
    float *sc = reinterpret_cast<float *>(sb + (((uint32_t)(npmax / 8) * L::kGroup + 127) & ~127u));
    uint32_t *shi = reinterpret_cast<uint32_t *>(sc + (scent ? (size_t)kmax * D : 0));
    uint32_t *slo = shi + (size_t)kmax * DS;
    int32_t *scnt = reinterpret_cast<int32_t *>(slo + (size_t)kmax * DS);

    if (tid == 0) {
        s_fail = 0;
        s_stat[0] = 0u;
        s_stat[1] = 0u;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (sacc) {
        for (int e = tid; e < kmax * DS; e += kTcThreads) {
            shi[e] = 0u;
            slo[e] = 0u;
        }
        for (int j = tid; j < kmax; j += kTcThreads) scnt[j] = 0;
    }
    if (warp == 0 && ub < ue) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"((uint32_t)nbuf * ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    if (ub >= ue) return;
    const uint32_t tmem = tmem_slot;
    uint32_t uses[2] = {0u, 0u};
    uint32_t issued[2] = {0u, 0u};
    uint32_t n_tie = 0, n_live = 0;

    for (int u = ub; u < ue;) {
        const int s = t.unit_seg[u];
        int ur = u + 1;
        while (ur < ue && t.unit_seg[ur] == s) ur++;
        const int k = t.k_eff[s];
        const int np = (k + 15) & ~15;                             // MMA N
        const int64_t c0 = t.cen_off[s];
        const int64_t row0 = t.seg_start[s] + t.unit_start[u];
        const int R = t.unit_start[ur - 1] + t.unit_count[ur - 1] - t.unit_start[u];
        u = ur;

        // ---- set-up of the run: float32 centers (for the near-tie re-scoring), reference
        // point (mean of the centers), operand B, cmax
        if (scent)
            for (int e = tid; e < k * D; e += kTcThreads) sc[e] = __ldg(&centers[c0 * D + e]);
        const float *cen = scent ? sc : centers + c0 * D;       // this set's centers
        {
            constexpr int G = kTcThreads / D;
            const int a = tid % D, g = tid / D;
            float m = 0.0f;
            if (g < G)
                for (int j = g; j < k; j += G) m = __fadd_rn(m, __ldg(&centers[(c0 + j) * D + a]));
            s_part[tid] = m;
            if (tid == 0) s_cmax2 = 0.0f;
            __syncthreads();
            if (tid < D) {
                float tot = 0.0f;
                for (int q = 0; q < G; q++) tot = __fadd_rn(tot, s_part[q * D + tid]);
                s_ref[tid] = __fdiv_rn(tot, (float)k);
            }
            __syncthreads();
        }
        for (int j = tid; j < np; j += kTcThreads) {
            float H[D], Lo[D], n2 = 0.0f;
#pragma unroll
            for (int a = 0; a < D; a++) {
                const float cc = j < k ? __fsub_rn(__ldg(&centers[(c0 + j) * D + a]), s_ref[a]) : 0.0f;
                n2 = __fmaf_rn(cc, cc, n2);
                const float m2 = -2.0f * cc;                          // exact
                H[a] = O::rnd(m2);
                Lo[a] = O::rnd(__fsub_rn(m2, H[a]));
            }
            float np_[O::kNormParts];
            {
                float rem = n2;
#pragma unroll
                for (int q = 0; q < O::kNormParts; q++) {
                    np_[q] = j < k ? O::rnd(rem) : 0.0f;
                    rem = __fsub_rn(rem, np_[q]);
                }
            }
            put_row<D, MODE>(sb, j, [&](int e) -> float {
                if (e < D) return H[e];
                if (O::kTerms == 3) {
                    if (e < 2 * D) return Lo[e - D];
                    if (e < 3 * D) return H[e - 2 * D];
                }
                const int q = e - O::kTerms * D;
                return q < O::kNormParts ? np_[q] : 0.0f;
            });
            if (j < k) atomicMax(reinterpret_cast<int *>(&s_cmax2), __float_as_int(n2));   // non-negative floats
        }
        __syncthreads();
        const uint32_t idesc = O::idesc(np);
        const float cmax = sqrtf(s_cmax2);
        // error bound of v_j (factor 2 margin): products (eta_p each, the -2 counted), float32
        // accumulation over K terms (2^-22 of the magnitude sum per term, allowing for
        // non-IEEE accumulation), centring (2^-24 per operand), norm parts and their sum
        const float alpha = 2.0f * (2.0f * O::eta_p() + 2.0f * (float)L::kK * 0x1p-22f + 0x1p-22f);
        const float beta = 2.0f * ((float)L::kK * 0x1p-22f + (float)(D + 4) * 0x1p-24f + 0x1p-22f);
        const int ntiles = (R + kTileRows - 1) / kTileRows;

        // rows of the next tile to stage, loaded one tile ahead (D <= 32: registers)
        constexpr bool kPre = D <= 32;
        float xp[kPre ? D : 1];
        auto load_rows = [&](int tile) {
            if (!kPre || tile >= ntiles) return;
            const int p = tile * kTileRows + tid;
            const float4 *x4 = reinterpret_cast<const float4 *>(pts + (row0 + (p < R ? p : 0)) * D);
#pragma unroll
            for (int a4 = 0; a4 < (kPre ? D : 4) / 4; a4++) {
                const float4 v = __ldg(&x4[a4]);
                xp[4 * a4 + 0] = v.x;
                xp[4 * a4 + 1] = v.y;
                xp[4 * a4 + 2] = v.z;
                xp[4 * a4 + 3] = v.w;
            }
        };
        // write tile `tile`'s A operand into buffer `buf` (threads = rows)
        auto stage = [&](int tile, int buf) {
            const int p = tile * kTileRows + tid;
            const bool live = p < R;
            const float4 *x4 = reinterpret_cast<const float4 *>(pts + (row0 + (live ? p : 0)) * D);
            float h[D], l[D];
#pragma unroll
            for (int a4 = 0; a4 < D / 4; a4++) {
                float vv[4];
                if (kPre) {
#pragma unroll
                    for (int q = 0; q < 4; q++) vv[q] = xp[(4 * a4 + q) % (kPre ? D : 1)];
                } else {
                    const float4 v = __ldg(&x4[a4]);
                    vv[0] = v.x;
                    vv[1] = v.y;
                    vv[2] = v.z;
                    vv[3] = v.w;
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int a = 4 * a4 + q;
                    const float xc = live ? __fsub_rn(vv[q], s_ref[a]) : 0.0f;
                    h[a] = O::rnd(xc);
                    l[a] = O::rnd(__fsub_rn(xc, h[a]));
                }
            }
            put_row<D, MODE>(sa0 + buf * L::kABytes, tid, [&](int e) { return a_elem<D, MODE>(e, h, l, live); });
            load_rows(tile + 1);           // in flight while this tile's MMAs and epilogue run
        };
        auto issue = [&](int buf) {
            issue_mma<D, MODE>(tmem + (uint32_t)buf * ncols, smem_u32(sa0 + buf * L::kABytes), smem_u32(sb), idesc,
                               smem_u32(&mbar[buf]));
        };
        auto stage_issue = [&](int tile, int buf) -> bool {
            stage(tile, buf);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (s_fail) return false;
            if (tid == 0) issue(buf);
            issued[buf]++;
            return true;
        };

        load_rows(0);
        bool ok = ntiles == 0 || stage_issue(0, 0);
        for (int i = 0; ok && i < ntiles; i++) {
            const int buf = nbuf == 2 ? (i & 1) : 0;
            // two deep: the next tile's MMAs run while this tile's epilogue does
            if (nbuf == 2 && i + 1 < ntiles && !stage_issue(i + 1, buf ^ 1)) break;
            if (!mbar_wait(smem_u32(&mbar[buf]), uses[buf] & 1u)) s_fail = 1;
            uses[buf]++;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            __syncthreads();
            if (s_fail) break;

            // ---- epilogue: this thread's row is TMEM lane tid of region `buf`
            const int p = i * kTileRows + tid;
            const bool live = p < R;
            const float4 *x4 = reinterpret_cast<const float4 *>(pts + (row0 + (live ? p : 0)) * D);
            float xv[D], xn2 = 0.0f;
#pragma unroll
            for (int a4 = 0; a4 < D / 4; a4++) {
                const float4 v = __ldg(&x4[a4]);
                xv[4 * a4 + 0] = v.x;
                xv[4 * a4 + 1] = v.y;
                xv[4 * a4 + 2] = v.z;
                xv[4 * a4 + 3] = v.w;
            }
#pragma unroll
            for (int a = 0; a < D; a++) {
                const float xc = __fsub_rn(xv[a], s_ref[a]);
                xn2 = __fmaf_rn(xc, xc, xn2);
            }
            const uint32_t trow = tmem + (uint32_t)buf * ncols + ((uint32_t)(warp * 32) << 16);
            // pass 1: the smallest v_j (four independent chains)
            const float kInf = __int_as_float(0x7f800000);
            float m4[4] = {kInf, kInf, kInf, kInf};
            for (int cb = 0; cb < k; cb += 32) {
                float v[32];
                tmem_ld32(trow + (uint32_t)cb, v);
#pragma unroll
                for (int q = 0; q < 32; q++) m4[q & 3] = fminf(m4[q & 3], cb + q < k ? v[q] : kInf);
            }
            const float best = fminf(fminf(m4[0], m4[1]), fminf(m4[2], m4[3]));
            // E bounds the error of every v_j; the float32 direct sums have their own error
            // (<= (d+3) 2^-24 of a distance, at most (||x~|| + cmax)^2), added so that no center
            // left out could win the float32 direct comparison
            const float xn = sqrtf(xn2);
            const float E = alpha * xn * cmax + beta * cmax * cmax +
                            (float)(2 * (D + 3)) * 0x1p-24f * (xn + cmax) * (xn + cmax) + 0x1p-100f;
            const float thr = best + 2.0f * E;
            // pass 2: every center within 2E of the best (the best among them), as a list of
            // 8-bit indices (k <= 256), in ascending index
            unsigned long long cl = 0ull;
            int nc = 0;
            for (int cb = 0; cb < k; cb += 32) {
                float v[32];
                tmem_ld32(trow + (uint32_t)cb, v);
#pragma unroll
                for (int q = 0; q < 32; q++) {
                    if (cb + q < k && v[q] <= thr) {
                        if (nc < 8) cl |= (unsigned long long)(cb + q) << (8 * nc);
                        nc++;
                    }
                }
            }
            int bj = (int)(cl & 0xFFu);
            const bool tie = live && nc > 1;
            if (__any_sync(0xffffffffu, tie)) {
                // near tie: re-score the candidates with the float32 direct sum, lowest index
                // among equal sums (the float32 path's choice); past 8 candidates, all centers
                auto direct = [&](int j) {
                    const float *cj = cen + (size_t)j * D;
                    float dd = 0.0f;
#pragma unroll
                    for (int a = 0; a < D; a++) {
                        const float tq = __fsub_rn(xv[a], cj[a]);      // shared or global (generic)
                        dd = __fmaf_rn(tq, tq, dd);
                    }
                    return dd;
                };
                const int nlist = tie ? (nc <= 8 ? nc : k) : 0;
                const int nmax = __reduce_max_sync(0xffffffffu, (unsigned)nlist);
                float bd = kInf;
                int bjj = bj;
                for (int c = 0; c < nmax; c++) {
                    if (c < nlist) {
                        const int j = nc <= 8 ? (int)((cl >> (8 * c)) & 0xFFu) : c;
                        const float dd = direct(j);
                        if (dd < bd) {                     // ascending j: strict keeps the lowest
                            bd = dd;
                            bjj = j;
                        }
                    }
                }
                if (tie) bj = bjj;
            }
            n_tie += tie;
            n_live += live;
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            if (live) {
                const int64_t row = row0 + p;
                labels[row] = bj;
                if (trace) trace[trace_off + row] = bj;
                if (sacc) {
                    atomicAdd(&scnt[bj], 1);
                    const size_t e0 = (size_t)bj * DS;
#pragma unroll
                    for (int a = 0; a < D; a++) {
                        const unsigned long long q = to_fix(xv[a]);
                        atomicAdd(&shi[e0 + a], (uint32_t)(q >> 16));
                        atomicAdd(&slo[e0 + a], (uint32_t)(q & 0xFFFFu));
                    }
                } else {                           // sums too large for shared memory
                    atomicAdd(&count[c0 + bj], 1);
#pragma unroll
                    for (int a = 0; a < D; a++) atomicAdd(&acc[(c0 + bj) * D + a], to_fix(xv[a]));
                }
            }
            if (sacc && (i + 1) % kFoldTiles == 0 && i + 1 < ntiles) {
                __syncthreads();
                flush_sums(shi, slo, scnt, k, c0, acc, count, D);
            }
            // one deep: the next tile after this epilogue released TMEM and the A buffer
            if (nbuf == 1 && i + 1 < ntiles) {
                __syncthreads();
                if (!stage_issue(i + 1, 0)) break;
            }
        }
        __syncthreads();
        if (sacc) flush_sums(shi, slo, scnt, k, c0, acc, count, D);
        if (s_fail) break;
    }
    {   // statistics: rows re-scored in float32 / rows assigned here
        const uint32_t nt = __reduce_add_sync(0xffffffffu, n_tie);
        const uint32_t nl = __reduce_add_sync(0xffffffffu, n_live);
        if (lane == 0) {
            atomicAdd(&s_stat[0], nt);
            atomicAdd(&s_stat[1], nl);
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (s_stat[0]) atomicAdd(&flags[2], s_stat[0]);
        if (s_stat[1]) atomicAdd(&flags[3], s_stat[1]);
    }
    if (s_fail) {
        // a commit never arrived: report, and give the MMAs still in flight a bounded
        // grace period before the tensor memory is released
        if (tid == 0) atomicOr(&flags[1], 4u);
        for (int b = 0; b < 2; b++)
            if (uses[b] < issued[b]) mbar_wait(smem_u32(&mbar[b]), uses[b] & 1u);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)nbuf * ncols));
}

template <int D, int MODE>
size_t tc_smem_bytes(int kmax, int nbuf, bool sacc, bool scent = false)
{
    using L = TcLayout<D, MODE>;
    const int np = (kmax + 15) & ~15;
    const size_t b = ((size_t)(np / 8) * L::kGroup + 127) & ~(size_t)127;
    return (size_t)nbuf * L::kABytes + b + (scent ? (size_t)kmax * D * 4 : 0) +
           (sacc ? (size_t)kmax * (D | 1) * 4 * 2 + (size_t)kmax * 4 : 0) + 1024;
}

// Two operand buffers and TMEM regions (MMA of the next tile under the epilogue of this
// one) when two regions fit in 256 columns and two A buffers in shared memory, else one.
template <int D, int MODE>
int tc_nbuf(int kmax)
{
    if (tmem_cols((kmax + 15) & ~15) > 128) return 1;
    return tc_smem_bytes<D, MODE>(kmax, 2, false) <= kTcSmemMax ? 2 : 1;
}

template <int D, int MODE>
cudaError_t tc_dispatch(const LloydBuffers &b, const SegTable &t, int iter, int unit_lo, int unit_hi, int kmax,
                        uint32_t *flags, int sm_count, cudaStream_t st, KTimer *kt)
{
    const int nbuf = tc_nbuf<D, MODE>(kmax);
    const uint32_t ncols = tmem_cols((kmax + 15) & ~15);
    // exact sums in shared memory when they fit next to the operands (else global atomics),
    // then the float32 centers for the re-scoring when they fit too (else read through L1)
    const int sacc = tc_smem_bytes<D, MODE>(kmax, nbuf, true) <= kTcSmemMax;
    const int scent = tc_smem_bytes<D, MODE>(kmax, nbuf, sacc != 0, true) <= kTcSmemMax;
    const size_t smem = tc_smem_bytes<D, MODE>(kmax, nbuf, sacc != 0, scent != 0);
    auto kern = k_lloyd_assign_tc<D, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int32_t *split = nullptr;
    int grid = unit_hi - unit_lo;
    if (t.split && unit_lo == 0 && unit_hi == t.n_units) {
        // persistent: as many CTAs per SM as shared memory, registers and the 512 TMEM
        // columns allow (<= 4), counted here (the occupancy query answers 1 for this kernel)
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        int dev = 0, smem_sm = 0, reserved = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
            return e;
        if ((e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess)
            return e;
        const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + reserved);
        const int by_regs = 65536 / (((fa.numRegs + 7) & ~7) * kTcThreads);
        const int by_tmem = (int)(512 / ((uint32_t)nbuf * ncols));
        const int m = std::max(1, std::min(std::min(by_smem, by_regs), std::min(by_tmem, 4)));
        split = t.split + t.split_off[m];
        grid = m * sm_count;
    }
    kt->begin(st);
    kern<<<grid, kTcThreads, smem, st>>>(b.pts, t, split, unit_lo, b.centers, b.acc, b.count, b.labels, b.trace,
                                         (int64_t)iter * b.rows, kmax, nbuf, ncols, sacc, scent, flags);
    kt->end(PSCL_K_LLOYD_ASSIGN, st);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t tc_by_d(const LloydBuffers &b, const SegTable &t, int d, int iter, int unit_lo, int unit_hi, int kmax,
                    uint32_t *flags, int sm_count, cudaStream_t st, KTimer *kt)
{
    switch (d) {
    case 4: return tc_dispatch<4, MODE>(b, t, iter, unit_lo, unit_hi, kmax, flags, sm_count, st, kt);
    case 8: return tc_dispatch<8, MODE>(b, t, iter, unit_lo, unit_hi, kmax, flags, sm_count, st, kt);
    case 16: return tc_dispatch<16, MODE>(b, t, iter, unit_lo, unit_hi, kmax, flags, sm_count, st, kt);
    case 32: return tc_dispatch<32, MODE>(b, t, iter, unit_lo, unit_hi, kmax, flags, sm_count, st, kt);
    case 64: return tc_dispatch<64, MODE>(b, t, iter, unit_lo, unit_hi, kmax, flags, sm_count, st, kt);
    default: return cudaErrorInvalidValue;
    }
}

template <int MODE>
size_t smem_by_d(int d, int kmax)
{
    switch (d) {
    case 4: return tc_smem_bytes<4, MODE>(kmax, 1, false);
    case 8: return tc_smem_bytes<8, MODE>(kmax, 1, false);
    case 16: return tc_smem_bytes<16, MODE>(kmax, 1, false);
    case 32: return tc_smem_bytes<32, MODE>(kmax, 1, false);
    case 64: return tc_smem_bytes<64, MODE>(kmax, 1, false);
    default: return ~(size_t)0;
    }
}

int mode_of(int prec)
{
    switch (prec) {
    case PSCL_PREC_BF16: return kModeBf16;
    case PSCL_PREC_TF32X3: return kModeTf32x3;
    case PSCL_PREC_BF16X3: return kModeBf16x3;
    default: return kModeTf32;
    }
}

}  // namespace

// The tensor-core assignment serves d in {4, 8, 16, 32, 64}, at most 256 centers per set
// and sets whose operands fit in 200 KB of shared memory (the exact sums go to shared
// memory when they fit too, else straight to the global sums); every other case takes
// the float32 direct kernel (same labels).
bool tc_supported(int d, int kmax, int prec)
{
    if (kmax < 1 || kmax > 256) return false;
    size_t need;
    switch (mode_of(prec)) {
    case kModeBf16: need = smem_by_d<kModeBf16>(d, kmax); break;
    case kModeTf32x3: need = smem_by_d<kModeTf32x3>(d, kmax); break;
    case kModeBf16x3: need = smem_by_d<kModeBf16x3>(d, kmax); break;
    default: need = smem_by_d<kModeTf32>(d, kmax); break;
    }
    return need <= kTcSmemMax;
}

cudaError_t launch_lloyd_assign_tc(const LloydBuffers &b, const SegTable &t, int d, int iter, int unit_lo,
                                   int unit_hi, int kmax, int prec, uint32_t *flags, int sm_count, cudaStream_t st,
                                   KTimer *kt)
{
    if (unit_hi <= unit_lo) return cudaSuccess;
    switch (mode_of(prec)) {
    case kModeBf16: return tc_by_d<kModeBf16>(b, t, d, iter, unit_lo, unit_hi, kmax, flags, sm_count, st, kt);
    case kModeTf32x3: return tc_by_d<kModeTf32x3>(b, t, d, iter, unit_lo, unit_hi, kmax, flags, sm_count, st, kt);
    case kModeBf16x3: return tc_by_d<kModeBf16x3>(b, t, d, iter, unit_lo, unit_hi, kmax, flags, sm_count, st, kt);
    default: return tc_by_d<kModeTf32>(b, t, d, iter, unit_lo, unit_hi, kmax, flags, sm_count, st, kt);
    }
}

}  // namespace pscl
