// Lloyd assignment step on the 5th-generation tensor cores (tcgen05, sm_103a): the
// "nearest center" of §I for every point of every set, as a contraction.
//
// For a tile of 128 rows x and the k <= 256 centers c of their set, with coordinates
// centred on a per-set reference point r (x~ = x - r, c~ = c - r; distances unchanged),
//     v_j = ||c~_j||^2 - 2 x~ . c~_j        (= ||x - c_j||^2 - ||x~||^2)
// is accumulated in float32 in tensor memory.  Operand modes (pscl_prec):
//   TF32 / BF16       A = [x~ | 1 ...], B = [-2c~ | n parts]  (one product per attribute)
//   TF32X3 / BF16X3   x~ = h + l and -2c~ = H + L split into two parts of the type; the MMAs
//                     add h.H + h.L + l.H (error ~2^-21 / 2^-17 per product instead of
//                     ~2^-10 / 2^-8)
// where the n parts sum to ||c~_j||^2 (split so that they survive the operand rounding).
//
// Near ties.  |v_j - exact| <= E = alpha ||x~|| cmax + beta cmax^2 (operand rounding,
// float32 accumulation, centring and norm errors; cmax = max_j ||c~_j||), plus the float32
// error of a direct distance.  A row whose second-best v lies within 2E of its best could
// be won by another center in the float32 direct comparison of the PSCL_PREC_FP32 path;
// such a row is marked (bit 31 of its label) and re-decided by k_tc_sums with the float32
// direct sum over all centers, lowest index on ties.  Every other row's best is the float32
// direct winner, so the labels equal those of the float32 path in every mode.
//
// The assignment kernel is persistent (contiguous unit ranges per CTA) and warp-specialised:
//   * producer warp: one thread streams 128-row tiles of the float32 points into shared
//     memory with cp.async.bulk.tensor (a tensor map over the packed points, rows of d
//     floats, boxes of 128 rows x min(d, 32) attributes with the bank swizzle that fits);
//   * converter warps (128 threads, a row each): centre the row, split it into the mode's
//     parts and write operand A in the canonical K-major layout (8-row x 16-byte core
//     matrices, no swizzle), with ||x~|| for the epilogue; at the start of each set they
//     build operand B from the set's centers;
//   * MMA warp: one thread issues the tcgen05.mma of a tile into one of two TMEM
//     accumulators and commits them to mbarriers (operand A free, accumulator full);
//   * two epilogue warpgroups, one per accumulator: each thread reads its row's k values
//     with tcgen05.ld and keeps the best and second best; it writes the label.
// Stages are handed over with mbarriers; every wait is bounded and a wait that runs out
// aborts the CTA (after its copies and MMAs in flight have drained) and sets flags[1] bit 2.
// The exact centroid sums are a separate pass (k_tc_sums), so the epilogue does only the
// minimum.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "pscl_internal.cuh"

namespace pscl {
namespace {

constexpr int kTileRows = 128;            // MMA M, rows per tile
constexpr int kCvtWarp0 = 8;              // converter warps 8..11
constexpr int kProdWarp = 12;
constexpr int kMmaWarp = 13;
constexpr int kTcThreads = 14 * 32;
constexpr int kXStages = 2;               // float32 point tiles in flight (deeper rings measured no faster)
constexpr int kAStages = 2;               // operand A buffers
constexpr int kMeta = 8;                  // per-tile metadata ring (tiles in flight < kMeta)
constexpr unsigned kDefaultWait = 1u << 26;
constexpr size_t kTcSmemMax = 220 * 1024;
constexpr uint32_t kTieBit = 0x80000000u; // label of a row left to the float32 re-scoring

enum TcMode { kModeTf32 = 0, kModeBf16 = 1, kModeTf32x3 = 2, kModeBf16x3 = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// min(a, b, c) in one instruction (sm_100 and later)
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float m;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(a), "f"(b), "f"(c));
    return m;
}

// all ones if v <= thr, else 0
__device__ __forceinline__ uint32_t le_mask(float v, float thr)
{
    uint32_t s;
    asm("set.le.u32.f32 %0, %1, %2;" : "=r"(s) : "f"(v), "f"(thr));
    return s;
}

// ---------------------------------------------------------------- mbarriers
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(a), "r"(parity)
                 : "memory");
    return done != 0;
}

// Bounded wait for phase `parity` of the mbarrier at a.  Gives up when the CTA is aborting
// (*abort set) or after `limit` polls, which starts the abort.  Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, unsigned limit, volatile int *abort)
{
    for (unsigned it = 0;; it++) {
        if (mbar_try(a, parity)) return true;
        if ((it & 31u) == 31u) {
            if (*abort) return false;
            if (it > limit) {
                *abort = 1;
                return false;
            }
        }
    }
}

// The same wait during clean-up: no abort check, only the limit.
__device__ __forceinline__ void mbar_drain(uint32_t a, uint32_t parity, unsigned limit)
{
    for (unsigned it = 0; it <= limit; it++)
        if (mbar_try(a, parity)) return;
}

// The converter warps' named barrier (id 1, 128 threads), returning the AND of `ok` over them.
__device__ __forceinline__ bool cvt_bar_and(bool ok)
{
    uint32_t r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.and.pred q, 1, 128, p;\n"
                 " selp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(r)
                 : "r"((uint32_t)ok)
                 : "memory");
    return r != 0;
}

// CTAs of the assignment kernel per SM the register budget is set for: two for narrow
// points, whose per-tile work is short and whose pipeline latency a second CTA hides
template <int D>
__host__ __device__ constexpr int tc_min_blocks()
{
    return D <= 32 ? 2 : 1;
}

// ---------------------------------------------------------------- TMA
// One box of the tensor map (x = attribute, y = row) into shared memory at dst; the bytes
// complete a transaction on the mbarrier at mbar.  Coordinates: x is a multiple of 32
// attributes (128 bytes), so it meets the 16-byte rule of tiled copies.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

// ---------------------------------------------------------------- tensor memory
// Columns [c, c + 32) of this warp's lanes, without waiting: tmem_wait() makes them usable.
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __host__ __forceinline__ uint32_t tmem_cols(int np)
{
    return np <= 32 ? 32u : (np <= 64 ? 64u : (np <= 128 ? 128u : 256u));
}

// Shared-memory matrix descriptor: K-major, no swizzle (version bit 46 of sm_100+).
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

// ---------------------------------------------------------------- operand modes
template <int MODE>
struct Op {
    static constexpr bool kBf16 = MODE == kModeBf16 || MODE == kModeBf16x3;
    static constexpr bool kSplit = MODE >= kModeTf32x3;
    static constexpr int kBytes = kBf16 ? 2 : 4;
    static constexpr int kPerChunk = 16 / kBytes;          // elements per 16-byte core-matrix row
    static constexpr int kMmaK = kBf16 ? 16 : 8;           // K of one MMA instruction
    static constexpr int kNormParts = kBf16 ? 3 : 2;
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

// Operand rows: [first part (D) | second part (D, split modes) | ones / norm parts (kMmaK)].
template <int D, int MODE>
struct TcLayout {
    using O = Op<MODE>;
    static constexpr int kParts = O::kSplit ? 2 : 1;
    static constexpr int kK = kParts * D + O::kMmaK;          // elements per operand row
    static constexpr int kChunks = kK / O::kPerChunk;          // 16-byte core-matrix columns
    static constexpr uint32_t kGroup = kChunks * 128;          // bytes per 8-row group (SBO)
    static constexpr uint32_t kABytes = (kTileRows / 8) * kGroup;
    static constexpr int kXBoxCols = D < 32 ? D : 32;          // attributes per TMA box
    static constexpr int kXBoxes = D / kXBoxCols;
    static constexpr uint32_t kXBoxBytes = kTileRows * kXBoxCols * 4;
    static constexpr uint32_t kXBytes = kXBoxes * kXBoxBytes;
    // bank swizzle of the boxes: its span equals the box row (bytes), 16 .. 128
    static constexpr int kSwzMask = kXBoxCols * 4 == 128 ? 7 : kXBoxCols * 4 == 64 ? 3 : kXBoxCols * 4 == 32 ? 1 : 0;
};

// Byte offset of 16-byte chunk c of row r in a point box (rows of kXBoxCols floats) after
// the TMA bank swizzle: the chunk index is XORed with bits 7.. of the row's byte offset.
template <int D, int MODE>
__device__ __forceinline__ uint32_t xbox_off(int r, int c)
{
    using L = TcLayout<D, MODE>;
    const uint32_t o = (uint32_t)r * (L::kXBoxCols * 4) + (uint32_t)c * 16;
    return o ^ (((o >> 7) & (uint32_t)L::kSwzMask) << 4);
}

// Byte offset of element e of row r in a K-major operand without swizzle.
template <int D, int MODE>
__device__ __forceinline__ uint32_t op_off(int r, int e)
{
    using O = Op<MODE>;
    using L = TcLayout<D, MODE>;
    return (uint32_t)(r >> 3) * L::kGroup + (uint32_t)(e / O::kPerChunk) * 128 + (uint32_t)(r & 7) * 16 +
           (uint32_t)(e % O::kPerChunk) * O::kBytes;
}

// Write 4 consecutive elements (e0 % 4 == 0) of row r of an operand.
template <int D, int MODE>
__device__ __forceinline__ void put4(unsigned char *base, int r, int e0, float a, float b, float c, float d)
{
    using O = Op<MODE>;
    unsigned char *p = base + op_off<D, MODE>(r, e0);
    if (O::kBf16) {
        const uint32_t lo = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
                            ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
        const uint32_t hi = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(c)) |
                            ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(d)) << 16);
        *reinterpret_cast<uint2 *>(p) = make_uint2(lo, hi);
    } else {
        *reinterpret_cast<uint4 *>(p) = make_uint4(__float_as_uint(a), __float_as_uint(b), __float_as_uint(c),
                                                   __float_as_uint(d));
    }
}

// Four bfloat16 elements (e0 % 4 == 0) of row r of a bfloat16 operand, already packed in pairs.
template <int D, int MODE>
__device__ __forceinline__ void put4_bits(unsigned char *base, int r, int e0, uint32_t lo, uint32_t hi)
{
    *reinterpret_cast<uint2 *>(base + op_off<D, MODE>(r, e0)) = make_uint2(lo, hi);
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<const uint32_t *>(&v); }

// ---------------------------------------------------------------- the assignment kernel
// Per-tile data the converters hand to the epilogue (a ring of kMeta entries).
struct TileMeta {
    float xn[kTileRows];         // ||x~|| of each row
    float cmax;                  // max_j ||c~_j|| of the tile's set
    int k;                       // centers of the set
    int nvalid;                  // rows of the tile inside its run
    int pad;
    long long row0;              // packed row of the tile's first row
};

struct TcArgs {
    const float *centers;
    int32_t *labels;
    uint32_t *tmask;             // 8 words per row: a near tie's candidate centers
    SegTable t;
    const int32_t *split;        // CTA c serves the units [split[c], split[c + 1])
    uint32_t *flags;
    unsigned wait_limit;
    int stall;                   // test hook: wait once on a barrier nothing completes
    int npmax;                   // operand B rows (centers rounded up to 16)
    uint32_t ncols;              // TMEM columns of one accumulator
    // Search of a whole set in chunks of centers (ref_centers != NULL): the launch covers
    // one chunk (centers, the set of its runs); the reference point and the error bound's
    // center norm come from all ref_k centers, so that every chunk's values compare.  Each
    // row keeps a running state across the chunks' launches: m1 = the smallest chunk
    // minimum, c1 = its candidate (bit 31: that chunk held more than one value within
    // twice the bound of it), m2 = the smallest minimum of the other chunks.  The last
    // chunk labels a row whose candidate is certain (c1 alone, m2 beyond m1 + 2E) and lists
    // every other row in ties[1 ...] (ties[0] the count) for float32 re-scoring.
    const float *ref_centers = nullptr;
    int ref_k = 0;
    int chunk_first = 0;         // index of the chunk's first center in the set
    int first_chunk = 0, last_chunk = 0;
    float *st_m1 = nullptr, *st_m2 = nullptr;
    int32_t *st_c1 = nullptr;
    uint32_t *ties = nullptr;
};

// A run: consecutive units of one set in a CTA's range, streamed as 128-row tiles.
struct Run {
    int s, k;
    int64_t c0, row0;
    int R, ntiles;
};

__device__ __forceinline__ bool next_run(const SegTable &t, int &u, int ue, Run &run)
{
    if (u >= ue) return false;
    const int s = t.unit_seg[u];
    int ur = u + 1;
    while (ur < ue && t.unit_seg[ur] == s) ur++;
    run.s = s;
    run.k = t.k_eff[s];
    run.c0 = t.cen_off[s];
    run.row0 = t.seg_start[s] + t.unit_start[u];
    run.R = t.unit_start[ur - 1] + t.unit_count[ur - 1] - t.unit_start[u];
    run.ntiles = (run.R + kTileRows - 1) / kTileRows;
    u = ur;
    return true;
}

template <int D, int MODE>
__global__ void __launch_bounds__(kTcThreads, tc_min_blocks<D>()) k_tc_assign(const __grid_constant__ CUtensorMap xmap, const TcArgs p)
{
    using O = Op<MODE>;
    using L = TcLayout<D, MODE>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // [point tiles | operand A buffers | operand B | metadata ring], from a 1024-byte
    // boundary (the bank swizzle of the point boxes repeats every 8 rows of 128 bytes)
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *sx = smem;
    constexpr int XS = kXStages;
    unsigned char *sa = sx + (size_t)XS * L::kXBytes;
    unsigned char *sb = sa + kAStages * L::kABytes;
    TileMeta *meta = reinterpret_cast<TileMeta *>(sb + (size_t)(p.npmax / 8) * L::kGroup);
    __shared__ __align__(8) uint64_t bars[2 * kXStages + 2 * kAStages + 4 + 2 * kMeta + 1];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    __shared__ float s_ref[D];
    __shared__ float s_part[128];
    __shared__ float s_cmax2;
    __shared__ uint32_t s_stat[2];
    const uint32_t b0 = smem_u32(bars);
    auto XFULL = [&](int s) { return b0 + 8u * (uint32_t)s; };
    auto XEMPTY = [&](int s) { return b0 + 8u * (uint32_t)(kXStages + s); };
    auto AFULL = [&](int s) { return b0 + 8u * (uint32_t)(2 * kXStages + s); };
    auto AEMPTY = [&](int s) { return b0 + 8u * (uint32_t)(2 * kXStages + kAStages + s); };
    auto TFULL = [&](int s) { return b0 + 8u * (uint32_t)(2 * kXStages + 2 * kAStages + s); };
    auto TEMPTY = [&](int s) { return b0 + 8u * (uint32_t)(2 * kXStages + 2 * kAStages + 2 + s); };
    auto MFULL = [&](int s) { return b0 + 8u * (uint32_t)(2 * kXStages + 2 * kAStages + 4 + s); };
    auto MEMPTY = [&](int s) { return b0 + 8u * (uint32_t)(2 * kXStages + 2 * kAStages + 4 + kMeta + s); };
    const uint32_t STALL = b0 + 8u * (uint32_t)(2 * kXStages + 2 * kAStages + 4 + 2 * kMeta);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ub = p.split[blockIdx.x], ue = p.split[blockIdx.x + 1];
    const unsigned lim = p.wait_limit;
    volatile int *abort = &s_abort;

    if (tid == 0) {
        s_abort = 0;
        s_stat[0] = 0u;
        s_stat[1] = 0u;
        for (int s = 0; s < XS; s++) {
            mbar_init(XFULL(s), 1);
            mbar_init(XEMPTY(s), 4);
        }
        for (int s = 0; s < kAStages; s++) {
            mbar_init(AFULL(s), 4);
            mbar_init(AEMPTY(s), 1);
        }
        for (int s = 0; s < 2; s++) {
            mbar_init(TFULL(s), 1);
            mbar_init(TEMPTY(s), 4);
        }
        for (int s = 0; s < kMeta; s++) {
            mbar_init(MFULL(s), 4);
            mbar_init(MEMPTY(s), 4);
        }
        mbar_init(STALL, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0 && ub < ue) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(2u * p.ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ub >= ue) return;
    // test hook: a wait on a barrier that nothing completes runs out before any copy or
    // MMA is issued, and the CTA leaves through the abort path
    if (p.stall && tid == 0) mbar_wait(STALL, 0u, lim, abort);
    __syncthreads();
    const uint32_t tmem = tmem_slot;

    if (warp == kProdWarp) {
        // ---- producer: point tiles by TMA
        uint32_t issued = 0;
        if (lane == 0 && !*abort) {
            int u = ub;
            Run run;
            uint32_t i = 0;
            bool ok = true;
            while (ok && next_run(p.t, u, ue, run)) {
                for (int tt = 0; tt < run.ntiles; tt++, i++) {
                    const int s = (int)(i % (uint32_t)XS);
                    const uint32_t use = i / (uint32_t)XS;
                    if (use > 0 && !mbar_wait(XEMPTY(s), (use - 1) & 1u, lim, abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(XFULL(s), L::kXBytes);
                    for (int bx = 0; bx < L::kXBoxes; bx++)
                        tma_load_2d(smem_u32(sx + (size_t)s * L::kXBytes + (size_t)bx * L::kXBoxBytes), &xmap,
                                    bx * L::kXBoxCols, (int)(run.row0 + (int64_t)tt * kTileRows), XFULL(s));
                    issued = i + 1;
                }
            }
            if (*abort)   // copies still in flight land before the CTA leaves
                for (uint32_t j = issued > (uint32_t)XS ? issued - (uint32_t)XS : 0u; j < issued; j++)
                    mbar_drain(XFULL((int)(j % (uint32_t)XS)), (j / (uint32_t)XS) & 1u, lim);
        }
    } else if (warp == kMmaWarp) {
        // ---- MMA issue: one thread
        if (lane == 0 && !*abort) {
            int u = ub;
            Run run;
            uint32_t i = 0, issued = 0;
            bool ok = true;
            while (ok && next_run(p.t, u, ue, run)) {
                const int np = (run.k + 15) & ~15;
                const uint32_t idesc = O::idesc(np);
                for (int tt = 0; tt < run.ntiles; tt++, i++) {
                    const int a = (int)(i % kAStages), bfr = (int)(i & 1u);
                    if (!mbar_wait(AFULL(a), (i / kAStages) & 1u, lim, abort) ||
                        (i >= 2 && !mbar_wait(TEMPTY(bfr), ((i >> 1) - 1) & 1u, lim, abort))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dcol = tmem + (uint32_t)bfr * p.ncols;
                    const uint32_t abase = smem_u32(sa + (size_t)a * L::kABytes), bbase = smem_u32(sb);
                    // products: (A part, B part) blocks; the last pairs the ones with the norm parts
                    constexpr int kGroups = O::kSplit ? 4 : 2;
                    const int ga[4] = {0, 0, 1, L::kParts};
                    const int gb[4] = {0, 1, 0, L::kParts};
                    uint32_t accum = 0;
#pragma unroll
                    for (int g = 0; g < kGroups; g++) {
                        const int pa = g == kGroups - 1 ? L::kParts : ga[g];
                        const int pb = g == kGroups - 1 ? L::kParts : gb[g];
                        const int nk = g == kGroups - 1 ? 1 : D / O::kMmaK;
                        for (int kb = 0; kb < nk; kb++) {
                            const uint32_t ca = (uint32_t)((pa * D) / O::kPerChunk + 2 * kb) * 128u;
                            const uint32_t cb = (uint32_t)((pb * D) / O::kPerChunk + 2 * kb) * 128u;
                            const uint64_t ad = smem_desc(abase + ca, 128, L::kGroup);
                            const uint64_t bd = smem_desc(bbase + cb, 128, L::kGroup);
                            if (O::kBf16)
                                asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n"
                                             ::"r"(dcol), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                            else
                                asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                                             " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}\n"
                                             ::"r"(dcol), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                            accum = 1;
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 ::"r"(AEMPTY(a)));
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 ::"r"(TFULL(bfr)));
                    issued = i + 1;
                }
            }
            if (*abort)   // MMAs still in flight finish before TMEM is released
                for (uint32_t j = issued > 2 ? issued - 2 : 0u; j < issued; j++)
                    mbar_drain(TFULL((int)(j & 1u)), (j >> 1) & 1u, lim);
        }
    } else if (warp >= kCvtWarp0) {
        // ---- converters: operand B per set, operand A and ||x~|| per tile
        const int r = tid - kCvtWarp0 * 32;                 // 0..127: the tile row of this thread
        int u = ub;
        Run run;
        uint32_t i = 0;
        bool ok = !*abort;
        // every converter thread passes the same named barriers: the set loop runs to the
        // end, and after a failed wait only the bookkeeping goes on
        while (next_run(p.t, u, ue, run)) {
            // the earlier tiles' MMAs must be done before operand B and s_ref change
            for (uint32_t j = i > kAStages ? i - kAStages : 0u; ok && j < i; j++)
                ok = mbar_wait(AEMPTY((int)(j % kAStages)), (j / kAStages) & 1u, lim, abort);
            ok = cvt_bar_and(ok && !*abort);
            if (!ok) {
                i += (uint32_t)run.ntiles;
                continue;
            }
            const int k = run.k, np = (k + 15) & ~15;
            const float *cen = p.centers + run.c0 * D;
            // the centers the reference point and the bound's center norm come from: the
            // set's (or, for a chunk of a whole-set search, all of the set's)
            const float *rcen = p.ref_centers ? p.ref_centers : cen;
            const int rk = p.ref_centers ? p.ref_k : k;
            {   // reference point: the mean of those centers
                constexpr int G = 128 / D;
                const int at = r % D, g = r / D;
                float m = 0.0f;
                if (g < G)
                    for (int j = g; j < rk; j += G) m = __fadd_rn(m, __ldg(&rcen[(size_t)j * D + at]));
                s_part[r] = m;
                if (r == 0) s_cmax2 = 0.0f;
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (r < D) {
                    float tot = 0.0f;
                    for (int q = 0; q < G; q++) tot = __fadd_rn(tot, s_part[q * D + r]);
                    s_ref[r] = __fdiv_rn(tot, (float)rk);
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");
            }
            if (p.ref_centers)       // the bound's center norm over the whole set
                for (int j = r; j < rk; j += 128) {
                    float n2 = 0.0f;
                    for (int a = 0; a < D; a++) {
                        const float c = __fsub_rn(__ldg(&rcen[(size_t)j * D + a]), s_ref[a]);
                        n2 = __fmaf_rn(c, c, n2);
                    }
                    atomicMax(reinterpret_cast<int *>(&s_cmax2), __float_as_int(n2));
                }
            // operand B: row j = [H | L | norm parts] of -2 c~_j (zero rows past k)
            for (int j = r; j < np; j += 128) {
                float n2 = 0.0f;
#pragma unroll 4
                for (int a4 = 0; a4 < D / 4; a4++) {
                    float4 c4 = j < k ? __ldg(reinterpret_cast<const float4 *>(cen + (size_t)j * D) + a4)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                    float cc[4] = {c4.x, c4.y, c4.z, c4.w}, H[4], Lo[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        cc[q] = j < k ? __fsub_rn(cc[q], s_ref[4 * a4 + q]) : 0.0f;
                        n2 = __fmaf_rn(cc[q], cc[q], n2);
                        const float m2 = -2.0f * cc[q];                 // exact
                        H[q] = O::rnd(m2);
                        Lo[q] = O::rnd(__fsub_rn(m2, H[q]));
                    }
                    put4<D, MODE>(sb, j, 4 * a4, H[0], H[1], H[2], H[3]);
                    if (O::kSplit) put4<D, MODE>(sb, j, D + 4 * a4, Lo[0], Lo[1], Lo[2], Lo[3]);
                }
                float np_[4] = {0.f, 0.f, 0.f, 0.f};
                {
                    float rem = n2;
#pragma unroll
                    for (int q = 0; q < O::kNormParts; q++) {
                        np_[q] = j < k ? O::rnd(rem) : 0.0f;
                        rem = __fsub_rn(rem, np_[q]);
                    }
                }
                put4<D, MODE>(sb, j, L::kParts * D, np_[0], np_[1], np_[2], np_[3]);
#pragma unroll
                for (int e = 4; e < O::kMmaK; e += 4) put4<D, MODE>(sb, j, L::kParts * D + e, 0.f, 0.f, 0.f, 0.f);
                if (j < k) atomicMax(reinterpret_cast<int *>(&s_cmax2), __float_as_int(n2));   // non-negative
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.sync 1, 128;" ::: "memory");
            const float cmax = sqrtf(s_cmax2);
            for (int tt = 0; tt < run.ntiles; tt++, i++) {
                const int xs = (int)(i % (uint32_t)XS), a = (int)(i % kAStages), m = (int)(i % kMeta);
                if (ok)
                    ok = mbar_wait(XFULL(xs), (i / (uint32_t)XS) & 1u, lim, abort) &&
                         (i < kAStages || mbar_wait(AEMPTY(a), (i / kAStages - 1) & 1u, lim, abort)) &&
                         (i < kMeta || mbar_wait(MEMPTY(m), (i / kMeta - 1) & 1u, lim, abort));
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) continue;
                const bool live = tt * kTileRows + r < run.R;
                const unsigned char *xt = sx + (size_t)xs * L::kXBytes;
                unsigned char *at = sa + (size_t)a * L::kABytes;
                float xn2 = 0.0f;
#pragma unroll 4
                for (int a4 = 0; a4 < D / 4; a4++) {
                    const int bx = (4 * a4) / L::kXBoxCols, c = ((4 * a4) % L::kXBoxCols) / 4;
                    const float4 v = *reinterpret_cast<const float4 *>(xt + (size_t)bx * L::kXBoxBytes +
                                                                       xbox_off<D, MODE>(r, c));
                    float xv[4] = {v.x, v.y, v.z, v.w}, xc[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        xc[q] = live ? __fsub_rn(xv[q], s_ref[4 * a4 + q]) : 0.0f;
                        xn2 = __fmaf_rn(xc[q], xc[q], xn2);
                    }
                    if constexpr (O::kBf16) {
                        // pairs rounded to bfloat16 in one conversion each, written as they are
                        const __nv_bfloat162 h01 = __floats2bfloat162_rn(xc[0], xc[1]);
                        const __nv_bfloat162 h23 = __floats2bfloat162_rn(xc[2], xc[3]);
                        put4_bits<D, MODE>(at, r, 4 * a4, bf2_bits(h01), bf2_bits(h23));
                        if (O::kSplit) {
                            const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
                            const __nv_bfloat162 l01 = __floats2bfloat162_rn(__fsub_rn(xc[0], f01.x), __fsub_rn(xc[1], f01.y));
                            const __nv_bfloat162 l23 = __floats2bfloat162_rn(__fsub_rn(xc[2], f23.x), __fsub_rn(xc[3], f23.y));
                            put4_bits<D, MODE>(at, r, D + 4 * a4, bf2_bits(l01), bf2_bits(l23));
                        }
                    } else {
                        float h[4], lo[4];
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            h[q] = O::rnd(xc[q]);
                            lo[q] = O::rnd(__fsub_rn(xc[q], h[q]));
                        }
                        put4<D, MODE>(at, r, 4 * a4, h[0], h[1], h[2], h[3]);
                        if (O::kSplit) put4<D, MODE>(at, r, D + 4 * a4, lo[0], lo[1], lo[2], lo[3]);
                    }
                }
                const float one = live ? 1.0f : 0.0f;
                put4<D, MODE>(at, r, L::kParts * D, one, one, O::kNormParts > 2 ? one : 0.0f, 0.0f);
#pragma unroll
                for (int e = 4; e < O::kMmaK; e += 4) put4<D, MODE>(at, r, L::kParts * D + e, 0.f, 0.f, 0.f, 0.f);
                meta[m].xn[r] = sqrtf(xn2);
                if (r == 0) {
                    meta[m].cmax = cmax;
                    meta[m].k = run.k;
                    meta[m].nvalid = min(kTileRows, run.R - tt * kTileRows);
                    meta[m].row0 = run.row0 + (int64_t)tt * kTileRows;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(XEMPTY(xs));
                    mbar_arrive(AFULL(a));
                    mbar_arrive(MFULL(m));
                }
            }
        }
    } else {
        // ---- epilogue warpgroup g = warp / 4 takes the tiles i with i % 2 == g
        const int g = warp >> 2, q4 = warp & 3, r = q4 * 32 + lane;
        const float kInf = __int_as_float(0x7f800000);
        constexpr int kTerms = (O::kSplit ? 3 : 1) * D + O::kMmaK;   // products accumulated per v_j
        // error bound of v_j (factor 2 margin): products (eta_p each, the -2 counted), float32
        // accumulation over the terms (2^-22 of the magnitude sum per term, allowing for
        // non-IEEE accumulation), centring (2^-24 per operand), norm parts and their sum
        const float alpha = 2.0f * (2.0f * O::eta_p() + 2.0f * (float)kTerms * 0x1p-22f + 0x1p-22f);
        const float beta = 2.0f * ((float)kTerms * 0x1p-22f + (float)(D + 4) * 0x1p-24f + 0x1p-22f);
        uint32_t n_tie = 0, n_row = 0;
        int u = ub;
        Run run;
        uint32_t i = 0;
        bool ok = !*abort;
        while (ok && next_run(p.t, u, ue, run)) {
            for (int tt = 0; tt < run.ntiles; tt++, i++) {
                if ((int)(i & 1u) != g) continue;
                const int m = (int)(i % kMeta);
                ok = mbar_wait(TFULL(g), (i >> 1) & 1u, lim, abort) && mbar_wait(MFULL(m), (i / kMeta) & 1u, lim, abort);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int k = meta[m].k;
                const float cmax = meta[m].cmax, xn = meta[m].xn[r];
                const bool live = r < meta[m].nvalid;
                const int64_t row = meta[m].row0 + r;
                const uint32_t taddr = tmem + (uint32_t)g * p.ncols + ((uint32_t)(q4 * 32) << 16);
                // pass 1: the smallest of the k values (four independent chains; two 32-column
                // loads in flight per wait)
                float m4[4] = {kInf, kInf, kInf, kInf};
                constexpr bool kLean = tc_min_blocks<D>() > 1;     // one load in flight: fewer registers
                constexpr int kStep = kLean ? 32 : 64;
                for (int cb = 0; cb < k; cb += kStep) {
                    uint32_t v0[32], v1[32];
                    const bool two = !kLean && cb + 32 < k;
                    tmem_ld32_nowait(taddr + (uint32_t)cb, v0);
                    if (two) tmem_ld32_nowait(taddr + (uint32_t)(cb + 32), v1);
                    tmem_wait();
                    if (cb + kStep <= k) {
#pragma unroll
                        for (int q = 0; q < 32; q += 2)
                            m4[(q >> 1) & 3] = min3f(m4[(q >> 1) & 3], __uint_as_float(v0[q]), __uint_as_float(v0[q + 1]));
                        if (!kLean) {
#pragma unroll
                            for (int q = 0; q < 32; q += 2)
                                m4[(q >> 1) & 3] =
                                    min3f(m4[(q >> 1) & 3], __uint_as_float(v1[q]), __uint_as_float(v1[q + 1]));
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 32; q++)
                            m4[q & 3] = fminf(m4[q & 3], cb + q < k ? __uint_as_float(v0[q]) : kInf);
                        if (two) {
#pragma unroll
                            for (int q = 0; q < 32; q++)
                                m4[q & 3] = fminf(m4[q & 3], cb + 32 + q < k ? __uint_as_float(v1[q]) : kInf);
                        }
                    }
                }
                const float b1 = fminf(fminf(m4[0], m4[1]), fminf(m4[2], m4[3]));
                // E bounds the error of every v_j; the float32 direct sums have their own error
                // (<= (d+3) 2^-24 of a distance, at most (||x~|| + cmax)^2), added so that no
                // center left out could win the float32 direct comparison
                const float E = alpha * xn * cmax + beta * cmax * cmax +
                                (float)(2 * (D + 3)) * 0x1p-24f * (xn + cmax) * (xn + cmax) + 0x1p-100f;
                const float thr = b1 + 2.0f * E;
                // pass 2: the centers with v_j <= thr as a bit mask (word c: centers 32c .. 32c+31);
                // one bit is the label, more a near tie
                uint32_t w[8];
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    w[c] = 0u;
                    if (32 * c < k) {
                        uint32_t v[32], acc = 0u;
                        tmem_ld32_nowait(taddr + (uint32_t)(32 * c), v);
                        tmem_wait();
#pragma unroll
                        for (int q = 0; q < 32; q++) acc |= le_mask(__uint_as_float(v[q]), thr) & (1u << q);
                        const int rem = k - 32 * c;          // columns past k hold no center
                        w[c] = rem >= 32 ? acc : acc & ((1u << rem) - 1u);
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(TEMPTY(g));
                int nc = 0, first = 0;
#pragma unroll
                for (int c = 7; c >= 0; c--) {
                    nc += __popc(w[c]);
                    if (w[c]) first = 32 * c + __ffs(w[c]) - 1;
                }
                if (p.ref_centers) {
                    // a chunk of a whole-set search: fold this chunk into the row's state
                    bool tie_row = false;
                    if (live) {
                        const int32_t cand = (p.chunk_first + first) | (nc > 1 ? (int32_t)kTieBit : 0);
                        float m1 = b1, m2 = kInf;
                        int32_t c1 = cand;
                        if (!p.first_chunk) {
                            m1 = p.st_m1[row];
                            m2 = p.st_m2[row];
                            c1 = p.st_c1[row];
                            if (b1 < m1) {
                                m2 = fminf(m2, m1);
                                m1 = b1;
                                c1 = cand;
                            } else {
                                m2 = fminf(m2, b1);
                            }
                        }
                        if (p.last_chunk) {
                            const bool unique = !((uint32_t)c1 & kTieBit) && m2 > m1 + 2.0f * E;
                            p.labels[row] = unique ? c1 : (int32_t)kTieBit;
                            tie_row = !unique;
                        } else {
                            p.st_m1[row] = m1;
                            p.st_m2[row] = m2;
                            p.st_c1[row] = c1;
                        }
                    }
                    if (p.last_chunk) {      // the rows left for float32 re-scoring, listed
                        const uint32_t bm = __ballot_sync(0xffffffffu, tie_row);
                        uint32_t base = 0;
                        if (lane == 0 && bm) base = atomicAdd(&p.ties[0], (uint32_t)__popc(bm));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (tie_row) p.ties[1 + base + __popc(bm & ((1u << lane) - 1u))] = (uint32_t)row;
                    }
                } else if (live) {
                    p.labels[row] = nc > 1 ? (int32_t)kTieBit : first;
                    if (nc > 1) {        // the candidates, for the sums pass to re-score
                        uint4 *mk = reinterpret_cast<uint4 *>(p.tmask + (size_t)row * 8);
                        mk[0] = make_uint4(w[0], w[1], w[2], w[3]);
                        mk[1] = make_uint4(w[4], w[5], w[6], w[7]);
                    }
                    n_tie += nc > 1;
                    n_row++;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(MEMPTY(m));
            }
        }
        const uint32_t nt = __reduce_add_sync(0xffffffffu, n_tie);
        const uint32_t nr = __reduce_add_sync(0xffffffffu, n_row);
        if (lane == 0) {
            atomicAdd(&s_stat[0], nt);
            atomicAdd(&s_stat[1], nr);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
        if (s_stat[0]) atomicAdd(&p.flags[2], s_stat[0]);
        if (s_stat[1]) atomicAdd(&p.flags[3], s_stat[1]);
        if (s_abort) atomicOr(&p.flags[1], 4u);
    }
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * p.ncols));
}

// ---------------------------------------------------------------- sums and near ties
// After the tensor-core assignment a warp re-scores each near-tie row against the candidate
// centers the assignment marked for it (those within twice the error bound of the best)
// with PSCL_PREC_FP32's arithmetic -- t = RN(x_a - c_a), acc = RN(t t + acc) in ascending a,
// the lowest index among equal sums -- so the label is the float32 direct winner.  Then each
// row's coordinates are added to its center's exact 32.32 fixed-point sum (a warp takes its
// rows a few at a time, lane a attribute a), as two 32-bit
// halves in shared memory (hi, lo <= 2^16 per row from fix_parts, so 32768 rows fit before
// a fold), folded into the 64-bit global sums at the end of each run of one set.
// Persistent: CTA c serves the units [split[c], split[c + 1]).  Also writes the final
// labels and the label trace.
constexpr int kFoldRows = 32768;

template <int D>
__host__ __device__ constexpr int sum_threads()
{
    return D <= 64 ? 512 : 256;          // a near tie's row is held in registers
}

template <int D>
__global__ void __launch_bounds__(sum_threads<D>(), D <= 32 ? 2 : 1) k_tc_sums(const float *__restrict__ pts,
                                                             const float *__restrict__ centers, SegTable t,
                                                             const int32_t *split, int32_t *labels,
                                                             const uint32_t *__restrict__ tmask,
                                                             int32_t *trace, int64_t trace_off,
                                                             unsigned long long *acc, int32_t *count, int kmax)
{
    constexpr int NT = sum_threads<D>();
    constexpr int DS = D | 1;            // odd stride: lanes adding one attribute of different centers spread over banks
    extern __shared__ uint32_t sm[];
    uint32_t *shi = sm;
    uint32_t *slo = shi + (size_t)kmax * DS;
    int32_t *scnt = reinterpret_cast<int32_t *>(slo + (size_t)kmax * DS);
    constexpr int DC = D + 4;            // centers' stride: float4 rows on distinct banks per quarter warp
    float *scen = reinterpret_cast<float *>(sm + ((2 * (size_t)kmax * DS + (size_t)kmax + 3) & ~(size_t)3));
    const int tid = threadIdx.x;
    const int ub = split[blockIdx.x], ue = split[blockIdx.x + 1];
    int u = ub;
    Run run;
    while (next_run(t, u, ue, run)) {
        const int k = run.k;
        const float *cen = centers + run.c0 * D;
        for (int e = tid; e < k * DS; e += NT) {
            shi[e] = 0u;
            slo[e] = 0u;
        }
        for (int j = tid; j < k; j += NT) scnt[j] = 0;
        for (int e = tid; e < k * D; e += NT) scen[(e / D) * DC + e % D] = __ldg(&cen[e]);
        __syncthreads();
        for (int p0 = 0; p0 < run.R; p0 += NT) {
            const int pr = p0 + tid;
            const bool live = pr < run.R;
            const int64_t row = run.row0 + (live ? pr : 0);
            int32_t lab = live ? labels[row] : 0;
            const bool tie = live && ((uint32_t)lab & kTieBit);
            if (!tie && (uint32_t)lab >= (uint32_t)k) lab = 0;   // only after an assignment that gave up
            // near ties: lane i of a warp re-scores the warp's i-th tie row against the row's
            // candidate centers (the bits of its mask; every center left out lies beyond the
            // float32 direct sum's error of the best), the centers read from shared memory as
            // float4 at a stride of D + 4 floats; the labels go back by shuffles
            {
                const int lane = tid & 31;
                const uint32_t tm = __ballot_sync(0xffffffffu, tie);
                if (tm) {
                    const int nt = __popc(tm);
                    const int src = lane < nt ? (int)__fns(tm, 0u, lane + 1) : 0;
                    const int64_t trow = __shfl_sync(0xffffffffu, row, src);
                    int32_t mylab = 0;
                    if (lane < nt) {
                        float x[D];
                        const float4 *x4 = reinterpret_cast<const float4 *>(pts + trow * D);
#pragma unroll
                        for (int a4 = 0; a4 < D / 4; a4++) {
                            const float4 v = __ldg(&x4[a4]);
                            x[4 * a4 + 0] = v.x;
                            x[4 * a4 + 1] = v.y;
                            x[4 * a4 + 2] = v.z;
                            x[4 * a4 + 3] = v.w;
                        }
                        const uint4 *mk = reinterpret_cast<const uint4 *>(tmask + trow * 8);
                        const uint4 ma = __ldg(mk), mb = __ldg(mk + 1);
                        uint32_t wd[8] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w};
#pragma unroll
                        for (int c = 0; c < 8; c++) {      // no bit at or past k
                            const int rem = k - 32 * c;
                            wd[c] &= rem >= 32 ? 0xffffffffu : rem > 0 ? (1u << rem) - 1u : 0u;
                        }
                        // the candidates in ascending order, two at a time (two independent
                        // chains); strict comparisons in that order keep the lowest index
                        // (the words move down as they empty: registers, no indexed access)
                        int base = 0, left = 8;
                        auto next = [&](int &j) -> bool {
                            while (wd[0] == 0u && left > 1) {
#pragma unroll
                                for (int q = 0; q < 7; q++) wd[q] = wd[q + 1];
                                wd[7] = 0u;
                                base += 32;
                                left--;
                            }
                            if (wd[0] == 0u) return false;
                            j = base + __ffs(wd[0]) - 1;
                            wd[0] &= wd[0] - 1u;
                            return true;
                        };
                        float bd = __int_as_float(0x7f800000);
                        int j0, j1;
                        while (next(j0)) {
                            const bool two = next(j1);
                            if (!two) j1 = j0;
                            const float4 *c0 = reinterpret_cast<const float4 *>(scen + (size_t)j0 * DC);
                            const float4 *c1 = reinterpret_cast<const float4 *>(scen + (size_t)j1 * DC);
                            float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
                            for (int a4 = 0; a4 < D / 4; a4++) {
                                const float4 u = c0[a4], w4 = c1[a4];
                                float t, y;
                                t = __fsub_rn(x[4 * a4 + 0], u.x); d0 = __fmaf_rn(t, t, d0);
                                y = __fsub_rn(x[4 * a4 + 0], w4.x); d1 = __fmaf_rn(y, y, d1);
                                t = __fsub_rn(x[4 * a4 + 1], u.y); d0 = __fmaf_rn(t, t, d0);
                                y = __fsub_rn(x[4 * a4 + 1], w4.y); d1 = __fmaf_rn(y, y, d1);
                                t = __fsub_rn(x[4 * a4 + 2], u.z); d0 = __fmaf_rn(t, t, d0);
                                y = __fsub_rn(x[4 * a4 + 2], w4.z); d1 = __fmaf_rn(y, y, d1);
                                t = __fsub_rn(x[4 * a4 + 3], u.w); d0 = __fmaf_rn(t, t, d0);
                                y = __fsub_rn(x[4 * a4 + 3], w4.w); d1 = __fmaf_rn(y, y, d1);
                            }
                            if (d0 < bd) {
                                bd = d0;
                                mylab = j0;
                            }
                            if (two && d1 < bd) {
                                bd = d1;
                                mylab = j1;
                            }
                        }
                    }
                    // the q-th tie lane of the warp gets the label lane q found
                    const int q = __popc(tm & ((1u << lane) - 1u));
                    const int32_t res = __shfl_sync(0xffffffffu, mylab, q);
                    if (tie) lab = res;
                }
            }
            if (live) {
                labels[row] = lab;
                if (trace) trace[trace_off + row] = lab;
                atomicAdd(&scnt[lab], 1);
            }
            // sums, RPI rows at a time per warp (lane a adds attribute a % D of row a / D; for
            // D >= 32 one row, lane a attributes a, a + 32, ...), so an atomic instruction
            // touches consecutive words of one center per row (no bank conflicts within a row)
            // and the rows are read in coalesced pieces
            {
                const int lane = tid & 31;
                const int64_t wrow0 = run.row0 + p0 + (tid & ~31);
                const int nrows = min(32, run.R - (p0 + (tid & ~31)));
                constexpr int RPI = D < 32 ? 32 / D : 1;       // rows per instruction
                constexpr int PL = D < 32 ? 1 : D / 32;        // attributes per lane
                constexpr int NI = 32 / RPI;                   // instructions per 32 rows
                const int sub = D < 32 ? lane / D : 0, at0 = D < 32 ? lane % D : lane;
                // the warp's 32 rows are all loaded before the first atomic
                float xv[NI][PL];
#pragma unroll
                for (int r = 0; r < NI; r++)
#pragma unroll
                    for (int e = 0; e < PL; e++) {
                        const int rr = r * RPI + sub;
                        xv[r][e] = rr < nrows ? __ldg(&pts[(wrow0 + rr) * D + at0 + 32 * e]) : 0.0f;
                    }
#pragma unroll
                for (int r = 0; r < NI; r++) {
                    const int rr = r * RPI + sub;
                    const int lr = __shfl_sync(0xffffffffu, lab, rr);
                    if (rr < nrows) {
#pragma unroll
                        for (int e = 0; e < PL; e++) {
                            uint32_t hi, lo;
                            fix_parts(xv[r][e], hi, lo);
                            atomicAdd(&shi[(size_t)lr * DS + at0 + 32 * e], hi);
                            atomicAdd(&slo[(size_t)lr * DS + at0 + 32 * e], lo);
                        }
                    }
                }
            }
            const bool fold = (p0 + NT) % kFoldRows == 0 || p0 + NT >= run.R;
            if (fold) {
                __syncthreads();
                for (int e = tid; e < k * D; e += NT) {
                    const int c = e / D, es = c * DS + (e - c * D);
                    const unsigned long long v = ((unsigned long long)shi[es] << 16) + slo[es];
                    if (v) atomicAdd(&acc[run.c0 * D + e], v);
                    shi[es] = 0u;
                    slo[es] = 0u;
                }
                for (int j = tid; j < k; j += NT) {
                    if (scnt[j]) atomicAdd(&count[run.c0 + j], scnt[j]);
                    scnt[j] = 0;
                }
                __syncthreads();
            }
        }
    }
}

// ---------------------------------------------------------------- whole-set search: ties, SSE
// The rows a whole-set search (the SSE pass) could not decide: a warp per row, lane l the
// centers l, l + 32, ..., with PSCL_PREC_FP32's arithmetic (t = RN(x_a - c_a), acc =
// RN(t t + acc) in ascending a; the lowest index among equal sums), so the label is the
// float32 direct winner.
template <int D>
__global__ void __launch_bounds__(256) k_tc_rescore_ties(const float *__restrict__ x, const float *__restrict__ centers,
                                                         int k, int32_t *labels, const uint32_t *ties)
{
    const uint32_t nt = __ldcg(&ties[0]);
    const int lane = threadIdx.x & 31;
    const uint32_t nw = gridDim.x * (blockDim.x / 32);
    for (uint32_t q = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; q < nt; q += nw) {
        const int64_t row = __ldcg(&ties[1 + q]);
        float xr[D];
        const float4 *x4 = reinterpret_cast<const float4 *>(x + row * D);
#pragma unroll
        for (int a4 = 0; a4 < D / 4; a4++) {
            const float4 v = __ldg(&x4[a4]);               // the same address in every lane
            xr[4 * a4 + 0] = v.x;
            xr[4 * a4 + 1] = v.y;
            xr[4 * a4 + 2] = v.z;
            xr[4 * a4 + 3] = v.w;
        }
        float bd = __int_as_float(0x7f800000);
        int bj = 0x7fffffff;
        for (int j = lane; j < k; j += 32) {
            const float4 *c4 = reinterpret_cast<const float4 *>(centers + (size_t)j * D);
            float acc = 0.0f;
#pragma unroll
            for (int a4 = 0; a4 < D / 4; a4++) {
                const float4 u = __ldg(&c4[a4]);
                float t;
                t = __fsub_rn(xr[4 * a4 + 0], u.x); acc = __fmaf_rn(t, t, acc);
                t = __fsub_rn(xr[4 * a4 + 1], u.y); acc = __fmaf_rn(t, t, acc);
                t = __fsub_rn(xr[4 * a4 + 2], u.z); acc = __fmaf_rn(t, t, acc);
                t = __fsub_rn(xr[4 * a4 + 3], u.w); acc = __fmaf_rn(t, t, acc);
            }
            if (acc < bd) {                                // ascending j in the lane
                bd = acc;
                bj = j;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float od = __shfl_xor_sync(0xffffffffu, bd, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (od < bd || (od == bd && oj < bj)) {
                bd = od;
                bj = oj;
            }
        }
        if (lane == 0) labels[row] = (uint32_t)bj < (uint32_t)k ? bj : 0;
    }
}

// The SSE from the labels: each point's float32 direct distance to its center, added in
// double per thread, per block in a fixed tree and over blocks in block order -- the rows of
// a thread, the tree and the block order of the float32 SSE pass (same grid, 256 threads),
// so the value is the same bit for bit.
template <int D>
__global__ void __launch_bounds__(256) k_sse_from_labels(const float *__restrict__ x, int64_t n,
                                                         const float *__restrict__ centers, int k,
                                                         const int32_t *__restrict__ labels, double *blk_sse,
                                                         double *sse, uint32_t *ticket)
{
    constexpr int NT = 256;
    double part = 0.0;
    const int64_t stride = (int64_t)gridDim.x * NT;
    const int64_t nround = (n + stride - 1) / stride;
    for (int64_t it = 0; it < nround; it++) {
        const int64_t i = it * stride + (int64_t)blockIdx.x * NT + threadIdx.x;
        if (i < n) {
            int32_t l = labels[i];
            if ((uint32_t)l >= (uint32_t)k) l = 0;          // only after a search that gave up
            const float *xr = x + i * D, *cr = centers + (size_t)l * D;
            float acc = 0.0f;
#pragma unroll
            for (int a = 0; a < D; a++) {
                const float t = __fsub_rn(__ldg(&xr[a]), __ldg(&cr[a]));
                acc = __fmaf_rn(t, t, acc);
            }
            part = __dadd_rn(part, (double)acc);
        }
    }
    for (int o = 16; o; o >>= 1) part = __dadd_rn(part, __shfl_down_sync(0xffffffffu, part, o));
    __shared__ double ws[NT / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = ws[0];
        for (int w = 1; w < NT / 32; w++) b = __dadd_rn(b, ws[w]);
        blk_sse[blockIdx.x] = b;
    }
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last || threadIdx.x != 0) return;
    __threadfence();
    double tot = 0.0;
    for (unsigned b = 0; b < gridDim.x; b++) tot = __dadd_rn(tot, __ldcg(&blk_sse[b]));
    *sse = tot;
    *ticket = 0;
}

// ---------------------------------------------------------------- host side
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver the runtime uses (looked up once, thread-safe).
EncodeTiled encode_tiled()
{
    static const EncodeTiled fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        cudaGetLastError();
        return reinterpret_cast<EncodeTiled>(f);
    }();
    return fn;
}

// The points' tensor map: rows of D floats, boxes of 128 rows x kXBoxCols attributes with
// the bank swizzle whose span is the box row.  Checked here before any launch: a base
// address and a row stride on 16-byte boundaries, box sizes within 256 elements and a box
// row that is a multiple of 16 bytes.
template <int D, int MODE>
cudaError_t make_xmap(const float *pts, int64_t rows, CUtensorMap *map)
{
    using L = TcLayout<D, MODE>;
    static_assert((L::kXBoxCols * 4) % 16 == 0 && L::kXBoxCols <= 256, "TMA box row");
    if (((uintptr_t)pts & 15u) != 0 || (D * 4) % 16 != 0 || rows < 1 || rows >= ((int64_t)1 << 32))
        return cudaErrorInvalidValue;
    EncodeTiled enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)D * 4};
    const cuuint32_t box[2] = {(cuuint32_t)L::kXBoxCols, (cuuint32_t)kTileRows};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle sw = L::kXBoxCols * 4 == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : L::kXBoxCols * 4 == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                  : L::kXBoxCols * 4 == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                           : CU_TENSOR_MAP_SWIZZLE_NONE;
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(pts), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int D, int MODE>
size_t assign_smem(int kmax)
{
    using L = TcLayout<D, MODE>;
    const int np = (kmax + 15) & ~15;
    return 1024 + (size_t)kXStages * L::kXBytes + (size_t)kAStages * L::kABytes + (size_t)(np / 8) * L::kGroup +
           (size_t)kMeta * sizeof(TileMeta);
}

template <int D>
size_t sums_smem(int kmax)
{
    return ((((size_t)2 * kmax * (D | 1) + (size_t)kmax + 3) & ~(size_t)3) + (size_t)kmax * (D + 4)) * 4;
}

template <int D, int MODE>
cudaError_t tc_dispatch(const LloydBuffers &b, const SegTable &t, int iter, int kmax, uint32_t *flags, int sm_count,
                        cudaStream_t st, KTimer *kt)
{
    CUtensorMap map;
    cudaError_t e = make_xmap<D, MODE>(b.pts, b.rows, &map);
    if (e != cudaSuccess) return e;
    TcArgs a;
    a.centers = b.centers;
    a.labels = b.labels;
    a.tmask = b.tmask;
    a.t = t;
    a.flags = flags;
    a.wait_limit = b.wait_limit ? b.wait_limit : kDefaultWait;
    a.stall = b.tc_stall;
    a.npmax = (kmax + 15) & ~15;
    a.ncols = tmem_cols(a.npmax);
    const size_t smem = assign_smem<D, MODE>(kmax);
    auto ka = k_tc_assign<D, MODE>;
    if ((e = cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    // as many CTAs per SM as registers, shared memory and the 512 TMEM columns allow (<= 4):
    // every resident CTA must get its TMEM at once
    int occ = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ka, kTcThreads, smem)) != cudaSuccess) return e;
    // d <= 32 is built for two CTAs per SM (at most 64 registers, under 80 KB of shared
    // memory each); the query answers one for it, but two CTAs' unit ranges run faster
    // (2^20 x 16: 1.70 -> 1.62 ms per job); no CTA waits on another, so the count is safe
    if (tc_min_blocks<D>() > 1) occ = std::max(occ, tc_min_blocks<D>());
    const int ma = std::max(1, std::min(std::min(occ, (int)(512u / (2u * a.ncols))), 4));
    a.split = t.split + t.split_off[ma];
    kt->begin(st);
    ka<<<ma * sm_count, kTcThreads, smem, st>>>(map, a);
    kt->end(PSCL_K_LLOYD_ASSIGN, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // sums: four CTAs' unit ranges per SM whatever fits at once, so that the block scheduler
    // evens out ranges whose near ties cost more
    const size_t ss = sums_smem<D>(kmax);
    auto ks = k_tc_sums<D>;
    if ((e = cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss)) != cudaSuccess) return e;
    const int m = 4;
    kt->begin(st);
    ks<<<m * sm_count, sum_threads<D>(), ss, st>>>(b.pts, b.centers, t, t.split + t.split_off[m], b.labels,
                                                   b.tmask, b.trace, (int64_t)iter * b.rows, b.acc, b.count, kmax);
    kt->end(PSCL_K_LLOYD_SUMS, st);
    return cudaGetLastError();
}

// A whole-set search on the tensor cores: the k centers in chunks of up to 256, one
// assignment launch per chunk (rows keep their running state), then the undecided rows
// re-scored in float32.  Leaves every row's float32 direct label in labels.
template <int D, int MODE>
cudaError_t chunk_search(const float *x, int64_t n, const float *centers, int k, const SegTable &t256,
                         const SegTable &trem, uint32_t *scratch, int32_t *labels, uint32_t *flags,
                         unsigned wait_limit, int sm_count, cudaStream_t st, KTimer *kt, int ktag)
{
    CUtensorMap map;
    cudaError_t e = make_xmap<D, MODE>(x, n, &map);
    if (e != cudaSuccess) return e;
    float *m1 = reinterpret_cast<float *>(scratch);
    float *m2 = m1 + n;
    int32_t *c1 = reinterpret_cast<int32_t *>(m2 + n);
    uint32_t *ties = reinterpret_cast<uint32_t *>(c1 + n);
    if ((e = cudaMemsetAsync(ties, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
    auto ka = k_tc_assign<D, MODE>;
    const int nch = (k + 255) / 256;
    for (int c = 0; c < nch; c++) {
        const int kc = std::min(256, k - 256 * c);
        const SegTable &t = kc == 256 ? t256 : trem;
        TcArgs a;
        a.centers = centers + (size_t)256 * c * D;
        a.labels = labels;
        a.tmask = nullptr;
        a.t = t;
        a.flags = flags;
        a.wait_limit = wait_limit ? wait_limit : kDefaultWait;
        a.stall = 0;
        a.npmax = (kc + 15) & ~15;
        a.ncols = tmem_cols(a.npmax);
        a.ref_centers = centers;
        a.ref_k = k;
        a.chunk_first = 256 * c;
        a.first_chunk = c == 0;
        a.last_chunk = c == nch - 1;
        a.st_m1 = m1;
        a.st_m2 = m2;
        a.st_c1 = c1;
        a.ties = ties;
        const size_t smem = assign_smem<D, MODE>(kc);
        if ((e = cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        int occ = 1;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ka, kTcThreads, smem)) != cudaSuccess) return e;
        const int ma = std::max(1, std::min(std::min(occ, (int)(512u / (2u * a.ncols))), 4));
        a.split = t.split + t.split_off[ma];
        kt->begin(st);
        ka<<<ma * sm_count, kTcThreads, smem, st>>>(map, a);
        kt->end(ktag, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    kt->begin(st);
    k_tc_rescore_ties<D><<<4 * sm_count, 256, 0, st>>>(x, centers, k, labels, ties);
    kt->end(ktag, st);
    return cudaGetLastError();
}

// The exact sums of one iteration from the labels, in global memory (sets too large for a
// CTA's shared memory): a thread per row adds its 32.32 fixed-point coordinates and its
// count with 64-bit atomics (integer sums: the order does not matter); writes the trace.
template <int D>
__global__ void __launch_bounds__(256) k_tc_global_sums(const float *__restrict__ pts, int64_t rows,
                                                        const int32_t *__restrict__ labels, int k, int32_t *trace,
                                                        int64_t trace_off, unsigned long long *acc, int32_t *count)
{
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (int64_t)gridDim.x * blockDim.x) {
        int32_t l = labels[row];
        if ((uint32_t)l >= (uint32_t)k) l = 0;              // only after a search that gave up
        if (trace) trace[trace_off + row] = l;
        atomicAdd(&count[l], 1);
        const float4 *x4 = reinterpret_cast<const float4 *>(pts + row * D);
        unsigned long long *al = acc + (size_t)l * D;
#pragma unroll 4
        for (int a4 = 0; a4 < D / 4; a4++) {
            const float4 v = __ldg(&x4[a4]);
            atomicAdd(&al[4 * a4 + 0], fix_of(v.x));
            atomicAdd(&al[4 * a4 + 1], fix_of(v.y));
            atomicAdd(&al[4 * a4 + 2], fix_of(v.z));
            atomicAdd(&al[4 * a4 + 3], fix_of(v.w));
        }
    }
}

// The SSE pass on the tensor cores: the chunked search, then the SSE from the labels.
template <int D, int MODE>
cudaError_t sse_tc_dispatch(const float *x, int64_t n, const float *centers, int k, const SegTable &t256,
                            const SegTable &trem, uint32_t *scratch, int32_t *labels, double *blk_sse, double *sse,
                            uint32_t *ticket, uint32_t *flags, unsigned wait_limit, int sm_count, cudaStream_t st,
                            KTimer *kt)
{
    cudaError_t e = chunk_search<D, MODE>(x, n, centers, k, t256, trem, scratch, labels, flags, wait_limit, sm_count,
                                          st, kt, PSCL_K_FINAL_SSE);
    if (e != cudaSuccess) return e;
    kt->begin(st);
    k_sse_from_labels<D><<<sse_grid(n, sm_count), 256, 0, st>>>(x, n, centers, k, labels, blk_sse, sse, ticket);
    kt->end(PSCL_K_FINAL_SSE, st);
    return cudaGetLastError();
}

// One Lloyd iteration of a single set with more than 256 centers on the tensor cores: the
// chunked search, then the exact sums from the labels (the update follows separately).
template <int D, int MODE>
cudaError_t lloyd_chunks_dispatch(const LloydBuffers &b, int iter, int k, uint32_t *flags, int sm_count,
                                  cudaStream_t st, KTimer *kt)
{
    cudaError_t e = chunk_search<D, MODE>(b.pts, b.rows, b.centers, k, b.chunk256, b.chunkrem, b.chunk_scratch,
                                          b.labels, flags, b.wait_limit, sm_count, st, kt, PSCL_K_LLOYD_ASSIGN);
    if (e != cudaSuccess) return e;
    int64_t g = (b.rows + 255) / 256;
    if (g > (int64_t)sm_count * 8) g = (int64_t)sm_count * 8;
    kt->begin(st);
    k_tc_global_sums<D><<<(int)std::max<int64_t>(1, g), 256, 0, st>>>(b.pts, b.rows, b.labels, k, b.trace,
                                                                        (int64_t)iter * b.rows, b.acc, b.count);
    kt->end(PSCL_K_LLOYD_SUMS, st);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t lloyd_chunks_by_d(int d, const LloydBuffers &b, int iter, int k, uint32_t *flags, int sm_count,
                              cudaStream_t st, KTimer *kt)
{
    switch (d) {
    case 16: return lloyd_chunks_dispatch<16, MODE>(b, iter, k, flags, sm_count, st, kt);
    case 32: return lloyd_chunks_dispatch<32, MODE>(b, iter, k, flags, sm_count, st, kt);
    case 64: return lloyd_chunks_dispatch<64, MODE>(b, iter, k, flags, sm_count, st, kt);
    case 128: return lloyd_chunks_dispatch<128, MODE>(b, iter, k, flags, sm_count, st, kt);
    default: return cudaErrorInvalidValue;
    }
}

template <int MODE>
cudaError_t sse_tc_by_d(int d, const float *x, int64_t n, const float *centers, int k, const SegTable &t256,
                        const SegTable &trem, uint32_t *scratch, int32_t *labels, double *blk_sse, double *sse,
                        uint32_t *ticket, uint32_t *flags, unsigned wait_limit, int sm_count, cudaStream_t st,
                        KTimer *kt)
{
    switch (d) {
    case 16: return sse_tc_dispatch<16, MODE>(x, n, centers, k, t256, trem, scratch, labels, blk_sse, sse, ticket, flags, wait_limit, sm_count, st, kt);
    case 32: return sse_tc_dispatch<32, MODE>(x, n, centers, k, t256, trem, scratch, labels, blk_sse, sse, ticket, flags, wait_limit, sm_count, st, kt);
    case 64: return sse_tc_dispatch<64, MODE>(x, n, centers, k, t256, trem, scratch, labels, blk_sse, sse, ticket, flags, wait_limit, sm_count, st, kt);
    case 128: return sse_tc_dispatch<128, MODE>(x, n, centers, k, t256, trem, scratch, labels, blk_sse, sse, ticket, flags, wait_limit, sm_count, st, kt);
    default: return cudaErrorInvalidValue;
    }
}

template <int MODE>
cudaError_t tc_by_d(const LloydBuffers &b, const SegTable &t, int d, int iter, int kmax, uint32_t *flags,
                    int sm_count, cudaStream_t st, KTimer *kt)
{
    switch (d) {
    case 16: return tc_dispatch<16, MODE>(b, t, iter, kmax, flags, sm_count, st, kt);
    case 32: return tc_dispatch<32, MODE>(b, t, iter, kmax, flags, sm_count, st, kt);
    case 64: return tc_dispatch<64, MODE>(b, t, iter, kmax, flags, sm_count, st, kt);
    case 128: return tc_dispatch<128, MODE>(b, t, iter, kmax, flags, sm_count, st, kt);
    default: return cudaErrorInvalidValue;
    }
}

template <int MODE>
bool fits_by_d(int d, int kmax)
{
    switch (d) {
    case 16: return assign_smem<16, MODE>(kmax) <= kTcSmemMax && sums_smem<16>(kmax) <= kTcSmemMax;
    case 32: return assign_smem<32, MODE>(kmax) <= kTcSmemMax && sums_smem<32>(kmax) <= kTcSmemMax;
    case 64: return assign_smem<64, MODE>(kmax) <= kTcSmemMax && sums_smem<64>(kmax) <= kTcSmemMax;
    case 128: return assign_smem<128, MODE>(kmax) <= kTcSmemMax && sums_smem<128>(kmax) <= kTcSmemMax;
    default: return false;
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

// PSCL_PREC_TC: TF32x3 where its operands fit, else BF16x3.
int resolve_prec(int d, int kmax, int prec)
{
    if (prec != PSCL_PREC_TC) return prec;
    return fits_by_d<kModeTf32x3>(d, kmax) ? PSCL_PREC_TF32X3 : PSCL_PREC_BF16X3;
}

}  // namespace

// The tensor-core assignment serves d in {16, 32, 64, 128} and at most 256 centers per
// set whose operands, point tiles and sums fit in shared memory; every other case takes
// the float32 direct kernel (same labels).
bool tc_supported(int d, int kmax, int prec)
{
    if (kmax < 1 || kmax > 256 || !encode_tiled()) return false;
    switch (mode_of(resolve_prec(d, kmax, prec))) {
    case kModeBf16: return fits_by_d<kModeBf16>(d, kmax);
    case kModeTf32x3: return fits_by_d<kModeTf32x3>(d, kmax);
    case kModeBf16x3: return fits_by_d<kModeBf16x3>(d, kmax);
    default: return fits_by_d<kModeTf32>(d, kmax);
    }
}

bool tc_sse_supported(int d, int k, int prec)
{
    return k >= 1 && tc_supported(d, std::min(k, 256), prec) &&
           (k <= 256 || tc_supported(d, 256, prec));
}

cudaError_t launch_lloyd_chunks_tc(const LloydBuffers &b, int d, int iter, int k, int prec, uint32_t *flags,
                                   int sm_count, cudaStream_t st, KTimer *kt)
{
    switch (mode_of(resolve_prec(d, 256, prec))) {
    case kModeBf16: return lloyd_chunks_by_d<kModeBf16>(d, b, iter, k, flags, sm_count, st, kt);
    case kModeTf32x3: return lloyd_chunks_by_d<kModeTf32x3>(d, b, iter, k, flags, sm_count, st, kt);
    case kModeBf16x3: return lloyd_chunks_by_d<kModeBf16x3>(d, b, iter, k, flags, sm_count, st, kt);
    default: return lloyd_chunks_by_d<kModeTf32>(d, b, iter, k, flags, sm_count, st, kt);
    }
}

cudaError_t launch_final_sse_tc(const float *x, int64_t n, int d, const float *centers, int k, const SegTable &t256,
                                const SegTable &trem, uint32_t *scratch, int32_t *labels, double *blk_sse,
                                double *sse, uint32_t *ticket, int prec, uint32_t *flags, unsigned wait_limit,
                                int sm_count, cudaStream_t st, KTimer *kt)
{
    const int ck = std::min(k, 256);
    switch (mode_of(resolve_prec(d, ck, prec))) {
    case kModeBf16: return sse_tc_by_d<kModeBf16>(d, x, n, centers, k, t256, trem, scratch, labels, blk_sse, sse, ticket, flags, wait_limit, sm_count, st, kt);
    case kModeTf32x3: return sse_tc_by_d<kModeTf32x3>(d, x, n, centers, k, t256, trem, scratch, labels, blk_sse, sse, ticket, flags, wait_limit, sm_count, st, kt);
    case kModeBf16x3: return sse_tc_by_d<kModeBf16x3>(d, x, n, centers, k, t256, trem, scratch, labels, blk_sse, sse, ticket, flags, wait_limit, sm_count, st, kt);
    default: return sse_tc_by_d<kModeTf32>(d, x, n, centers, k, t256, trem, scratch, labels, blk_sse, sse, ticket, flags, wait_limit, sm_count, st, kt);
    }
}

cudaError_t launch_lloyd_assign_tc(const LloydBuffers &b, const SegTable &t, int d, int iter, int kmax, int prec,
                                   uint32_t *flags, int sm_count, cudaStream_t st, KTimer *kt)
{
    if (!t.split) return cudaErrorInvalidValue;
    switch (mode_of(resolve_prec(d, kmax, prec))) {
    case kModeBf16: return tc_by_d<kModeBf16>(b, t, d, iter, kmax, flags, sm_count, st, kt);
    case kModeTf32x3: return tc_by_d<kModeTf32x3>(b, t, d, iter, kmax, flags, sm_count, st, kt);
    case kModeBf16x3: return tc_by_d<kModeBf16x3>(b, t, d, iter, kmax, flags, sm_count, st, kt);
    default: return tc_by_d<kModeTf32>(b, t, d, iter, kmax, flags, sm_count, st, kt);
    }
}

}  // namespace pscl
