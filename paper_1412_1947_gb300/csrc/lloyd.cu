// Lloyd's k-means (§I) on many point sets at once: every subcluster of Algorithm 1
// step 4, and the pooled local centers of §V.
//
// Layout: the points of all sets are packed row-major one set after another (the
// paper's "flattening while subgrouping", §V); set s has seg_size[s] rows starting at
// seg_start[s] and k_eff[s] centers starting at cen_off[s] in one P x d center array.
// Work is cut into units of at most a few thousand rows of one set, so a launch keeps
// every SM busy whatever the mix of set sizes.
//
// One iteration = k_lloyd_assign (nearest center of every row, lowest index on ties,
// and the row's coordinates added to its center's sum) + k_lloyd_finalize (center =
// sum / count; an empty cluster keeps its center).  The sums are exact: coordinates
// (scaled to [0, 1]) are rounded once to 32.32 fixed point and added as 64-bit
// integers, first in shared memory, then with one global atomic per (center,
// attribute) and unit.  Integer addition is associative, so the result does not depend
// on how units are scheduled or batched with other work.
#include "pscl_internal.cuh"

namespace pscl {
namespace {

constexpr int kThreads = 256;
constexpr float kFix = 4294967296.0f;                  // 2^32
constexpr size_t kSmemAccMax = 96 * 1024;              // shared accumulators up to this size
constexpr int kCenterChunkBytes = 48 * 1024;           // center chunk held in shared memory

// ---------------------------------------------------------------- SplitMix64
// Steele, Lea & Flood (OOPSLA 2014): the state advances by the golden-ratio constant
// and each output is the variant-13 mix of the state.
__device__ __forceinline__ uint64_t sm64_next(uint64_t &s)
{
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Initial centers of set s: the first k positions of a Fisher-Yates shuffle of its m
// rows (step i swaps i with i + r mod (m - i)), the stream keyed by (seed, stage, s).
// Only positions < k and at most k others are ever touched, so the shuffle keeps a
// dense table for 0..k-1 and an open-addressing table for the rest.
__global__ void k_lloyd_init(const float *__restrict__ pts, SegTable t, int d, float *centers,
                             unsigned long long *acc, int32_t *count2, int64_t P,
                             uint64_t seed, uint32_t stage, int first_k)
{
    extern __shared__ int32_t sh[];
    for (int s = blockIdx.x; s < t.n_seg; s += gridDim.x) {
        const int k = t.k_eff[s];
        const int32_t m = t.seg_size[s];
        int cap = 1;
        while (cap < 2 * k) cap <<= 1;
        int32_t *A = sh;                       // k
        int32_t *hk = sh + k;                  // cap keys (-1 = empty)
        int32_t *hv = hk + cap;                // cap values
        for (int i = threadIdx.x; i < k; i += blockDim.x) A[i] = i;
        for (int i = threadIdx.x; i < cap; i += blockDim.x) hk[i] = -1;
        __syncthreads();
        if (threadIdx.x == 0 && !first_k) {
            uint64_t key = ((uint64_t)stage << 32) | (uint64_t)(uint32_t)s;
            uint64_t st = seed ^ sm64_next(key);
            for (int i = 0; i < k; i++) {
                uint64_t r = sm64_next(st);
                int32_t j = i + (int32_t)(r % (uint64_t)(m - i));
                if (j < k) {
                    int32_t tmp = A[i];
                    A[i] = A[j];
                    A[j] = tmp;
                } else {
                    uint32_t h = ((uint32_t)j * 0x9E3779B1u) & (uint32_t)(cap - 1);
                    while (hk[h] != -1 && hk[h] != j) h = (h + 1) & (uint32_t)(cap - 1);
                    int32_t vj = hk[h] == j ? hv[h] : j;
                    hk[h] = j;
                    hv[h] = A[i];
                    A[i] = vj;
                }
            }
        }
        __syncthreads();
        const int64_t row0 = t.seg_start[s];
        const int64_t c0 = t.cen_off[s];
        for (int e = threadIdx.x; e < k * d; e += blockDim.x) {
            int j = e / d, a = e - j * d;
            centers[(c0 + j) * d + a] = pts[(row0 + A[j]) * d + a];
            acc[(c0 + j) * d + a] = 0ull;
        }
        for (int j = threadIdx.x; j < k; j += blockDim.x) {
            count2[c0 + j] = 0;
            count2[P + c0 + j] = 0;
        }
        __syncthreads();
    }
}

// float32 direct squared distance, ascending attributes, one fused rounding per term.
template <int D>
__device__ __forceinline__ float dist_direct(const float *x, const float *c, int d)
{
    float acc = 0.0f;
    const int dd = D > 0 ? D : d;
#pragma unroll
    for (int j = 0; j < dd; j++) {
        float t = __fsub_rn(x[j], c[j]);
        acc = __fmaf_rn(t, t, acc);
    }
    return acc;
}

__device__ __forceinline__ unsigned long long to_fix(float v) { return fix_of(v); }

// Squared distances of R rows (registers) to one center (shared memory), float32
// direct form, ascending attributes; the center is read as float4 when D % 4 == 0.
template <int D, int R>
__device__ __forceinline__ void dist_rows(const float (&xv)[R][D], const float *c, float (&out)[R])
{
#pragma unroll
    for (int q = 0; q < R; q++) out[q] = 0.0f;
    if (D % 4 == 0) {
        const float4 *c4 = reinterpret_cast<const float4 *>(c);
#pragma unroll
        for (int j4 = 0; j4 < D / 4; j4++) {
            const float4 cv = c4[j4];
            const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
#pragma unroll
                for (int q = 0; q < R; q++) {
                    const float tq = __fsub_rn(xv[q][4 * j4 + e], cc[e]);
                    out[q] = __fmaf_rn(tq, tq, out[q]);
                }
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < D; j++) {
            const float cj = c[j];
#pragma unroll
            for (int q = 0; q < R; q++) {
                const float tq = __fsub_rn(xv[q][j], cj);
                out[q] = __fmaf_rn(tq, tq, out[q]);
            }
        }
    }
}

// One assignment step over work units [unit_lo, unit_lo + gridDim.x).
//   D > 0: d == D known at compile time, each thread keeps R rows in registers and
//          reads every center once for all of them; D == 0: any d, one row at a time.
template <int D, int R, bool kSmemAcc>
__global__ void __launch_bounds__(kThreads)
k_lloyd_assign(const float *__restrict__ pts, SegTable t, int d, const float *__restrict__ centers,
               unsigned long long *acc, int32_t *count, int32_t *labels, int32_t *trace,
               int64_t trace_off, int unit_lo, int chunk_k, const int32_t *__restrict__ weights)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int DR = D > 0 ? D : 1;
    const int u = unit_lo + blockIdx.x;
    const int s = t.unit_seg[u];
    const int k = t.k_eff[s];
    const int64_t c0 = t.cen_off[s];
    const int64_t row0 = t.seg_start[s] + t.unit_start[u];
    const int rows = t.unit_count[u];
    const int dd = D > 0 ? D : d;

    // [center chunk | high sums | low sums | counts], each 16-byte aligned.  A fixed-point
    // value q <= 2^32 is added as q >> 11 (<= 2^21) and q & 0x7FF with two native 32-bit
    // shared atomics; a unit has at most 1024 rows, so neither sum can wrap, and the
    // flush recombines them exactly into the 64-bit global sums.  A center's sums take an
    // odd stride ds = d | 1, so that the lanes of a warp adding attribute a of different
    // centers fall in different banks (with stride 16 they shared two).
    const int ds = dd | 1;
    const size_t c_bytes = ((size_t)min(chunk_k, k) * dd * 4 + 15) & ~(size_t)15;
    float *sc = reinterpret_cast<float *>(smem);
    uint32_t *shi = reinterpret_cast<uint32_t *>(smem + c_bytes);
    uint32_t *slo = shi + (size_t)k * ds;
    int32_t *scnt = reinterpret_cast<int32_t *>(slo + (size_t)k * ds);
    if (kSmemAcc) {
        for (int e = threadIdx.x; e < k * ds; e += kThreads) {
            shi[e] = 0u;
            slo[e] = 0u;
        }
        for (int j = threadIdx.x; j < k; j += kThreads) scnt[j] = 0;
    }
    const bool one_chunk = chunk_k >= k;
    if (one_chunk) {
        for (int e = threadIdx.x; e < k * dd; e += kThreads) sc[e] = centers[c0 * dd + e];
    }
    __syncthreads();

    for (int p0 = 0; p0 < rows; p0 += kThreads * R) {
        float xv[R][DR];
        bool live[R];
        int prow[R];
#pragma unroll
        for (int q = 0; q < R; q++) {
            prow[q] = p0 + q * kThreads + threadIdx.x;
            live[q] = prow[q] < rows;
            if (D > 0) {
                const float *xr = pts + (row0 + (live[q] ? prow[q] : 0)) * dd;
                if (D % 4 == 0) {
                    const float4 *x4 = reinterpret_cast<const float4 *>(xr);
#pragma unroll
                    for (int j4 = 0; j4 < DR / 4; j4++) {
                        const float4 v = __ldg(&x4[j4]);
                        xv[q][4 * j4 + 0] = v.x;
                        xv[q][4 * j4 + 1] = v.y;
                        xv[q][4 * j4 + 2] = v.z;
                        xv[q][4 * j4 + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < DR; j++) xv[q][j] = __ldg(&xr[j]);
                }
            }
        }
        float best[R];
        int bj[R];
#pragma unroll
        for (int q = 0; q < R; q++) {
            best[q] = __int_as_float(0x7f800000);
            bj[q] = 0;
        }
        for (int cb = 0; cb < k; cb += chunk_k) {
            const int ce = min(k, cb + chunk_k);
            if (!one_chunk) {
                __syncthreads();
                for (int e = threadIdx.x; e < (ce - cb) * dd; e += kThreads)
                    sc[e] = centers[(c0 + cb) * dd + e];
                __syncthreads();
            }
            const float *cbase = one_chunk ? sc + (size_t)cb * dd : sc;
            int j = cb;
            if constexpr (D > 0) {
                // two centers per step: two independent sets of chains in flight (3.6 %
                // faster at d = 64, where a thread keeps one row); the comparisons stay in
                // center order (lowest index on ties)
                for (; j + 1 < ce; j += 2) {
                    const float *cj = cbase + (size_t)(j - cb) * dd;
                    float v[R], w[R];
                    dist_rows<DR, R>(xv, cj, v);
                    dist_rows<DR, R>(xv, cj + dd, w);
#pragma unroll
                    for (int q = 0; q < R; q++) {
                        if (v[q] < best[q]) { best[q] = v[q]; bj[q] = j; }
                        if (w[q] < best[q]) { best[q] = w[q]; bj[q] = j + 1; }
                    }
                }
            }
            for (; j < ce; j++) {
                const float *cj = cbase + (size_t)(j - cb) * dd;
                float v[R];
                if (D > 0) {
                    dist_rows<DR, R>(xv, cj, v);
                } else {
                    const float *xr = pts + (row0 + (live[0] ? prow[0] : 0)) * dd;
                    v[0] = 0.0f;
                    for (int a = 0; a < dd; a++) {
                        const float tq = __fsub_rn(__ldg(&xr[a]), cj[a]);
                        v[0] = __fmaf_rn(tq, tq, v[0]);
                    }
                }
#pragma unroll
                for (int q = 0; q < R; q++)
                    if (v[q] < best[q]) { best[q] = v[q]; bj[q] = j; }
            }
        }
#pragma unroll
        for (int q = 0; q < R; q++) {
            if (!live[q]) continue;
            const int64_t row = row0 + prow[q];
            labels[row] = bj[q];
            if (trace) trace[trace_off + row] = bj[q];
            const float *xr = pts + row * dd;
            if (kSmemAcc) {
                atomicAdd(&scnt[bj[q]], 1);
                const size_t e0 = (size_t)bj[q] * ds;
                if (D > 0) {
#pragma unroll
                    for (int j = 0; j < DR; j++) {
                        const unsigned long long v = to_fix(xv[q][j]);
                        atomicAdd(&shi[e0 + j], (uint32_t)(v >> 11));
                        atomicAdd(&slo[e0 + j], (uint32_t)(v & 0x7FFu));
                    }
                } else {
                    for (int j = 0; j < dd; j++) {
                        const unsigned long long v = to_fix(__ldg(&xr[j]));
                        atomicAdd(&shi[e0 + j], (uint32_t)(v >> 11));
                        atomicAdd(&slo[e0 + j], (uint32_t)(v & 0x7FFu));
                    }
                }
            } else {
                // weighted rows (global sums only): w x and w; a zero weight adds nothing
                const unsigned long long w = weights ? (unsigned long long)(uint32_t)weights[row] : 1ull;
                if (w == 0ull) continue;
                atomicAdd(&count[c0 + bj[q]], (int)w);
                if (D > 0) {
#pragma unroll
                    for (int j = 0; j < DR; j++) atomicAdd(&acc[(c0 + bj[q]) * dd + j], to_fix(xv[q][j]) * w);
                } else {
                    for (int j = 0; j < dd; j++) atomicAdd(&acc[(c0 + bj[q]) * dd + j], to_fix(__ldg(&xr[j])) * w);
                }
            }
        }
    }
    if (kSmemAcc) {
        __syncthreads();
        for (int e = threadIdx.x; e < k * dd; e += kThreads) {
            const int c = e / dd, es = c * ds + (e - c * dd);
            const unsigned long long v = ((unsigned long long)shi[es] << 11) + slo[es];
            if (v) atomicAdd(&acc[c0 * dd + e], v);
        }
        for (int j = threadIdx.x; j < k; j += kThreads) {
            int v = scnt[j];
            if (v) atomicAdd(&count[c0 + j], v);
        }
    }
}

// center = exact sum / count (double), rounded once to float; empty clusters keep their
// center.  Clears the sums and the other parity's counts for the next iteration.  A thread
// takes EPT consecutive attributes of one center (d % EPT == 0) and forms the count's
// reciprocal once for them: float64 is the slow pipe of this GPU.  I is the element index
// type (32-bit whenever the elements fit, which avoids 64-bit division).
template <int EPT, typename I>
__global__ void k_lloyd_finalize(float *centers, unsigned long long *acc, const int32_t *count,
                                 int32_t *count_next, int64_t cen_lo, int64_t cen_hi, int d)
{
    const I g0 = (I)(cen_lo * d / EPT), g1 = (I)(cen_hi * d / EPT), dd = (I)d;
    for (I g = g0 + (I)blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += (I)gridDim.x * blockDim.x) {
        const I e = g * EPT;
        const I c = e / dd;
        const int32_t n = count[c];
        if (n > 0) {
            const double r = __drcp_rn((double)n);
#pragma unroll
            for (int q = 0; q < EPT; q++) {
                const long long sum = (long long)acc[e + q];
                centers[e + q] = __double2float_rn(__dmul_rn(__dmul_rn((double)sum, 0x1p-32), r));
            }
        }
#pragma unroll
        for (int q = 0; q < EPT; q++) acc[e + q] = 0ull;
        if (e - c * dd == 0) count_next[c] = 0;
    }
}

template <int EPT>
void finalize_launch(const LloydBuffers &b, int32_t *count_next, int64_t cen_lo, int64_t cen_hi, int d,
                     int sm_count, cudaStream_t st)
{
    const int64_t work = (cen_hi - cen_lo) * d / EPT;
    int64_t g = (work + 255) / 256;
    if (g > (int64_t)sm_count * 8) g = (int64_t)sm_count * 8;
    if (g < 1) g = 1;
    if (cen_hi * d < ((int64_t)1 << 31))
        k_lloyd_finalize<EPT, uint32_t><<<(int)g, 256, 0, st>>>(b.centers, b.acc, b.count, count_next, cen_lo, cen_hi, d);
    else
        k_lloyd_finalize<EPT, int64_t><<<(int)g, 256, 0, st>>>(b.centers, b.acc, b.count, count_next, cen_lo, cen_hi, d);
}

// Nearest final center of every scaled point (original order) and the sum of squared
// errors: each point's float32 direct distance is added in double, per thread, then
// per block in a fixed tree, then over blocks in block order.
template <int D>
__global__ void __launch_bounds__(kThreads)
k_final_sse(const float *__restrict__ x, int64_t n, int d, const float *__restrict__ centers,
            int k, int chunk_k, int32_t *labels, double *blk_sse, double *sse, uint32_t *ticket)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *sc = reinterpret_cast<float *>(smem);
    const int dd = D > 0 ? D : d;
    const bool one_chunk = chunk_k >= k;
    if (one_chunk) {
        for (int e = threadIdx.x; e < k * dd; e += kThreads) sc[e] = centers[e];
        __syncthreads();
    }
    double part = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    const int64_t nround = (n + stride - 1) / stride;
    for (int64_t it = 0; it < nround; it++) {
        const int64_t i = it * stride + (int64_t)blockIdx.x * kThreads + threadIdx.x;
        const bool live = i < n;
        const float *xr = x + (live ? i : 0) * dd;
        float xv[D > 0 ? D : 1];
        if (D > 0) {
#pragma unroll
            for (int j = 0; j < (D > 0 ? D : 1); j++) xv[j] = __ldg(&xr[j]);
        }
        const float *xp = D > 0 ? xv : xr;
        float best = __int_as_float(0x7f800000);
        int bj = 0;
        for (int cb = 0; cb < k; cb += chunk_k) {
            const int ce = min(k, cb + chunk_k);
            if (!one_chunk) {
                __syncthreads();
                for (int e = threadIdx.x; e < (ce - cb) * dd; e += kThreads) sc[e] = centers[(size_t)cb * dd + e];
                __syncthreads();
            }
            const float *cbase = one_chunk ? sc + (size_t)cb * dd : sc;
            if (live) {
                for (int j = cb; j < ce; j++) {
                    float v = dist_direct<D>(xp, cbase + (size_t)(j - cb) * dd, dd);
                    if (v < best) { best = v; bj = j; }
                }
            }
        }
        if (live) {
            labels[i] = bj;
            part = __dadd_rn(part, (double)best);
        }
    }
    // fixed-order block reduction
    for (int o = 16; o; o >>= 1) part = __dadd_rn(part, __shfl_down_sync(0xffffffffu, part, o));
    __shared__ double ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = ws[0];
        for (int w = 1; w < kThreads / 32; w++) b = __dadd_rn(b, ws[w]);
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

int center_chunk(int d, int k)
{
    int c = kCenterChunkBytes / (d * 4);
    if (c < 1) c = 1;
    return c >= k ? k : c;
}

// Per work unit of independent sets: the nearest center of every row among its set's
// centers (float32 direct form, lowest index on ties) and the sum of those squared
// distances in double (per thread in row order, then a fixed tree over the block).
template <int D>
__global__ void __launch_bounds__(kThreads)
k_seg_sse(const float *__restrict__ pts, SegTable t, int d, const float *__restrict__ centers, int chunk_k,
          int32_t *labels, double *unit_sse)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *sc = reinterpret_cast<float *>(smem);
    const int u = blockIdx.x;
    const int s = t.unit_seg[u];
    const int k = t.k_eff[s];
    const int64_t c0 = t.cen_off[s];
    const int64_t row0 = t.seg_start[s] + t.unit_start[u];
    const int rows = t.unit_count[u];
    const int dd = D > 0 ? D : d;
    double part = 0.0;
    for (int p0 = 0; p0 < rows; p0 += kThreads) {
        const int p = p0 + threadIdx.x;
        const bool live = p < rows;
        const float *xr = pts + (row0 + (live ? p : 0)) * dd;
        float xv[D > 0 ? D : 1];
        if (D > 0) {
#pragma unroll
            for (int j = 0; j < (D > 0 ? D : 1); j++) xv[j] = __ldg(&xr[j]);
        }
        const float *xp = D > 0 ? xv : xr;
        float best = __int_as_float(0x7f800000);
        int bj = 0;
        for (int cb = 0; cb < k; cb += chunk_k) {
            const int ce = min(k, cb + chunk_k);
            __syncthreads();
            for (int e = threadIdx.x; e < (ce - cb) * dd; e += kThreads) sc[e] = centers[(c0 + cb) * dd + e];
            __syncthreads();
            if (live) {
                for (int j = cb; j < ce; j++) {
                    const float v = dist_direct<D>(xp, sc + (size_t)(j - cb) * dd, dd);
                    if (v < best) { best = v; bj = j; }
                }
            }
        }
        if (live) {
            labels[row0 + p] = bj;
            part = __dadd_rn(part, (double)best);
        }
    }
    for (int o = 16; o; o >>= 1) part = __dadd_rn(part, __shfl_down_sync(0xffffffffu, part, o));
    __shared__ double ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = ws[0];
        for (int w = 1; w < kThreads / 32; w++) b = __dadd_rn(b, ws[w]);
        unit_sse[u] = b;
    }
}

// SSE of every set: its units' sums in unit order.
__global__ void k_seg_sse_fold(const double *unit_sse, const int32_t *seg_unit0, int n_seg, double *seg_sse)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_seg) return;
    double v = 0.0;
    for (int u = seg_unit0[s]; u < seg_unit0[s + 1]; u++) v = __dadd_rn(v, unit_sse[u]);
    seg_sse[s] = v;
}

template <int D>
cudaError_t seg_sse_dispatch(const float *pts, const SegTable &t, int d, const float *centers, int kmax,
                             int32_t *labels, double *unit_sse, cudaStream_t st, KTimer *kt)
{
    const int chunk = center_chunk(d, kmax);
    const size_t smem = (size_t)chunk * d * 4;
    auto kern = k_seg_sse<D>;
    if (const cudaError_t ea = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return ea;
    kt->begin(st);
    kern<<<t.n_units, kThreads, smem, st>>>(pts, t, d, centers, chunk, labels, unit_sse);
    kt->end(PSCL_K_FINAL_SSE, st);
    return cudaGetLastError();
}

// rows kept in registers per thread: 64 floats of rows at most
template <int D>
__host__ __device__ constexpr int kRowsPerThread()
{
    return D <= 0 ? 1 : (D >= 64 ? 1 : 64 / D > 4 ? 4 : 64 / D);
}

template <int D, int R>
cudaError_t assign_launch(const LloydBuffers &b, const SegTable &t, int d, int iter, int unit_lo,
                          int unit_hi, int kmax, cudaStream_t st, KTimer *kt)
{
    const int chunk = center_chunk(d, kmax);
    const size_t acc_bytes = (size_t)kmax * (d | 1) * 8 + (size_t)kmax * 4;
    const size_t c_bytes = ((size_t)chunk * d * 4 + 15) & ~(size_t)15;
    const bool smem_acc = !b.weights && acc_bytes <= kSmemAccMax;
    const size_t smem = (smem_acc ? acc_bytes : 0) + c_bytes;
    const int grid = unit_hi - unit_lo;
    if (grid <= 0) return cudaSuccess;
    if (smem_acc) {
        auto kern = k_lloyd_assign<D, R, true>;
        if (const cudaError_t ea = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return ea;
        kt->begin(st);
        kern<<<grid, kThreads, smem, st>>>(b.pts, t, d, b.centers, b.acc, b.count, b.labels, b.trace,
                                           (int64_t)iter * b.rows, unit_lo, chunk, b.weights);
        kt->end(PSCL_K_LLOYD_ASSIGN, st);
    } else {
        auto kern = k_lloyd_assign<D, R, false>;
        if (const cudaError_t ea = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return ea;
        kt->begin(st);
        kern<<<grid, kThreads, smem, st>>>(b.pts, t, d, b.centers, b.acc, b.count, b.labels, b.trace,
                                           (int64_t)iter * b.rows, unit_lo, chunk, b.weights);
        kt->end(PSCL_K_LLOYD_ASSIGN, st);
    }
    return cudaGetLastError();
}

// rows_per_thread: 0 = kRowsPerThread<D>(), 1 = one row per thread, 2 = eight rows per
// thread for d <= 16 (tuning choices; the result is the same)
template <int D>
cudaError_t assign_dispatch(const LloydBuffers &b, const SegTable &t, int d, int iter, int unit_lo,
                            int unit_hi, int kmax, int rows_per_thread, cudaStream_t st, KTimer *kt)
{
    if (rows_per_thread == 1 && kRowsPerThread<D>() > 1)
        return assign_launch<D, 1>(b, t, d, iter, unit_lo, unit_hi, kmax, st, kt);
    if (rows_per_thread == 2 && D > 0 && D <= 16)                 // 8 rows: half the center reads
        return assign_launch<D, (D > 0 && D <= 16 ? 8 : 1)>(b, t, d, iter, unit_lo, unit_hi, kmax, st, kt);
    return assign_launch<D, kRowsPerThread<D>()>(b, t, d, iter, unit_lo, unit_hi, kmax, st, kt);
}

template <int D>
cudaError_t sse_dispatch(const float *x, int64_t n, int d, const float *centers, int k, int32_t *labels,
                         double *blk_sse, double *sse, uint32_t *ticket, int sm_count, cudaStream_t st,
                         KTimer *kt)
{
    const int chunk = center_chunk(d, k);
    const size_t smem = (size_t)chunk * d * 4;
    int64_t want = (n + kThreads - 1) / kThreads;
    int grid = (int)(want < (int64_t)sm_count * 8 ? want : (int64_t)sm_count * 8);
    if (grid < 1) grid = 1;
    auto kern = k_final_sse<D>;
    if (const cudaError_t ea = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return ea;
    kt->begin(st);
    kern<<<grid, kThreads, smem, st>>>(x, n, d, centers, k, chunk, labels, blk_sse, sse, ticket);
    kt->end(PSCL_K_FINAL_SSE, st);
    return cudaGetLastError();
}

}  // namespace

int sse_grid(int64_t n, int sm_count)
{
    int64_t want = (n + kThreads - 1) / kThreads;
    return (int)(want < (int64_t)sm_count * 8 ? want : (int64_t)sm_count * 8);
}

cudaError_t launch_lloyd_init(const LloydBuffers &b, const SegTable &t, int d, int64_t P,
                              uint64_t seed, uint32_t stage, int first_k, int kmax, cudaStream_t st,
                              KTimer *kt)
{
    int cap = 1;
    while (cap < 2 * kmax) cap <<= 1;
    size_t smem = ((size_t)kmax + 2 * (size_t)cap) * sizeof(int32_t);
    if (const cudaError_t ea = cudaFuncSetAttribute(k_lloyd_init, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return ea;
    int grid = t.n_seg < 65535 ? t.n_seg : 65535;
    kt->begin(st);
    k_lloyd_init<<<grid, 256, smem, st>>>(b.pts, t, d, b.centers, b.acc, b.count, P, seed, stage, first_k);
    kt->end(PSCL_K_LLOYD_INIT, st);
    return cudaGetLastError();
}

// One Lloyd iteration over units [unit_lo, unit_hi) and centers [cen_lo, cen_hi).
// b.count must point at this iteration's count buffer; count_next at the other one.
cudaError_t launch_lloyd_iter(const LloydBuffers &b, int32_t *count_next, const SegTable &t, int d,
                              int iter, int unit_lo, int unit_hi, int64_t cen_lo, int64_t cen_hi,
                              int kmax, int prec, uint32_t *flags, int sm_count, cudaStream_t st,
                              KTimer *kt, int rows_per_thread)
{
    cudaError_t e;
    if (prec != PSCL_PREC_FP32 && !b.weights && b.tmask && t.split && unit_lo == 0 && unit_hi == t.n_units &&
        tc_supported(d, kmax, prec)) {
        e = launch_lloyd_assign_tc(b, t, d, iter, kmax, prec, flags, sm_count, st, kt);
    } else if (prec != PSCL_PREC_FP32 && !b.weights && b.has_chunks && b.chunk_scratch && t.n_seg == 1 &&
               kmax > 256 && unit_lo == 0 && unit_hi == t.n_units && tc_sse_supported(d, kmax, prec)) {
        e = launch_lloyd_chunks_tc(b, d, iter, kmax, prec, flags, sm_count, st, kt);
    } else switch (d) {
    case 2: e = assign_dispatch<2>(b, t, d, iter, unit_lo, unit_hi, kmax, rows_per_thread, st, kt); break;
    case 4: e = assign_dispatch<4>(b, t, d, iter, unit_lo, unit_hi, kmax, rows_per_thread, st, kt); break;
    case 8: e = assign_dispatch<8>(b, t, d, iter, unit_lo, unit_hi, kmax, rows_per_thread, st, kt); break;
    case 16: e = assign_dispatch<16>(b, t, d, iter, unit_lo, unit_hi, kmax, rows_per_thread, st, kt); break;
    case 32: e = assign_dispatch<32>(b, t, d, iter, unit_lo, unit_hi, kmax, rows_per_thread, st, kt); break;
    case 64: e = assign_dispatch<64>(b, t, d, iter, unit_lo, unit_hi, kmax, rows_per_thread, st, kt); break;
    case 128: e = assign_dispatch<128>(b, t, d, iter, unit_lo, unit_hi, kmax, rows_per_thread, st, kt); break;
    default: e = assign_dispatch<0>(b, t, d, iter, unit_lo, unit_hi, kmax, rows_per_thread, st, kt); break;
    }
    if (e != cudaSuccess) return e;
    kt->begin(st);
    if (d % 4 == 0) finalize_launch<4>(b, count_next, cen_lo, cen_hi, d, sm_count, st);
    else if (d % 2 == 0) finalize_launch<2>(b, count_next, cen_lo, cen_hi, d, sm_count, st);
    else finalize_launch<1>(b, count_next, cen_lo, cen_hi, d, sm_count, st);
    kt->end(PSCL_K_LLOYD_FINALIZE, st);
    return cudaGetLastError();
}

cudaError_t launch_seg_sse(const float *pts, const SegTable &t, const int32_t *seg_unit0, int d,
                           const float *centers, int kmax, int32_t *labels, double *unit_sse, double *seg_sse,
                           cudaStream_t st, KTimer *kt)
{
    cudaError_t e;
    switch (d) {
    case 2: e = seg_sse_dispatch<2>(pts, t, d, centers, kmax, labels, unit_sse, st, kt); break;
    case 4: e = seg_sse_dispatch<4>(pts, t, d, centers, kmax, labels, unit_sse, st, kt); break;
    case 8: e = seg_sse_dispatch<8>(pts, t, d, centers, kmax, labels, unit_sse, st, kt); break;
    case 16: e = seg_sse_dispatch<16>(pts, t, d, centers, kmax, labels, unit_sse, st, kt); break;
    case 32: e = seg_sse_dispatch<32>(pts, t, d, centers, kmax, labels, unit_sse, st, kt); break;
    case 64: e = seg_sse_dispatch<64>(pts, t, d, centers, kmax, labels, unit_sse, st, kt); break;
    case 128: e = seg_sse_dispatch<128>(pts, t, d, centers, kmax, labels, unit_sse, st, kt); break;
    default: e = seg_sse_dispatch<0>(pts, t, d, centers, kmax, labels, unit_sse, st, kt); break;
    }
    if (e != cudaSuccess) return e;
    k_seg_sse_fold<<<(t.n_seg + 255) / 256, 256, 0, st>>>(unit_sse, seg_unit0, t.n_seg, seg_sse);
    return cudaGetLastError();
}

cudaError_t launch_final_sse(const float *x, int64_t n, int d, const float *centers, int k,
                             int32_t *labels, double *blk_sse, double *sse, uint32_t *ticket,
                             int sm_count, cudaStream_t st, KTimer *kt)
{
    switch (d) {
    case 2: return sse_dispatch<2>(x, n, d, centers, k, labels, blk_sse, sse, ticket, sm_count, st, kt);
    case 4: return sse_dispatch<4>(x, n, d, centers, k, labels, blk_sse, sse, ticket, sm_count, st, kt);
    case 8: return sse_dispatch<8>(x, n, d, centers, k, labels, blk_sse, sse, ticket, sm_count, st, kt);
    case 16: return sse_dispatch<16>(x, n, d, centers, k, labels, blk_sse, sse, ticket, sm_count, st, kt);
    case 32: return sse_dispatch<32>(x, n, d, centers, k, labels, blk_sse, sse, ticket, sm_count, st, kt);
    case 64: return sse_dispatch<64>(x, n, d, centers, k, labels, blk_sse, sse, ticket, sm_count, st, kt);
    case 128: return sse_dispatch<128>(x, n, d, centers, k, labels, blk_sse, sse, ticket, sm_count, st, kt);
    default: return sse_dispatch<0>(x, n, d, centers, k, labels, blk_sse, sse, ticket, sm_count, st, kt);
    }
}

}  // namespace pscl
