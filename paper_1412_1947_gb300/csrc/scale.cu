// Feature scaling (Algorithm 1, step 1): min-max of every attribute to [0, 1].
//
//   mn_j = min_i x_ij, mx_j = max_i x_ij              (exact in any order)
//   x'_ij = RN( (double(x_ij) - mn_j) * (1 / (mx_j - mn_j)) )  in double, 0 if mx_j = mn_j,
//           rounded once to the storage type (float32, or bfloat16 kept in a float)
//
// Two kernels: a column min/max reduction (per-block partials, the last block to finish
// folds them) and an element-wise pass.  Both are HBM-bound (2 reads + 1 write of n*d*4
// bytes in total) once the element-wise pass avoids the float64 pipe, which is narrow on
// this GPU: it computes the product in float-float and falls back to float64 only where
// that cannot decide the rounding (scaled_value below).
#include <cuda_bf16.h>

#include <algorithm>
#include <numeric>

#include "pscl_internal.cuh"

namespace pscl {
namespace {

constexpr uint32_t kInfBits = 0x7f800000u;

// The last block of a reduction folds the gridDim.x per-block partials (exact in any
// order): with d <= blockDim.x, thread t folds attribute t mod d over blocks t / d,
// + blockDim.x / d, ..., then the threads of each attribute meet in shared memory (sm holds
// 2 blockDim.x floats); wider points fold one attribute per thread.
__device__ void fold_partials(const float *part, int d, float *sm, double *mn, double *mx)
{
    const int t = threadIdx.x, nb = (int)gridDim.x;
    if (d > (int)blockDim.x) {
        for (int a = t; a < d; a += blockDim.x) {
            float l = __int_as_float(kInfBits), h = -__int_as_float(kInfBits);
            for (int b = 0; b < nb; b++) {
                l = fminf(l, __ldcg(&part[(size_t)b * d + a]));
                h = fmaxf(h, __ldcg(&part[(size_t)(nb + b) * d + a]));
            }
            mn[a] = (double)l;
            mx[a] = (double)h;
        }
        return;
    }
    const int lanes = (int)blockDim.x / d;
    float l = __int_as_float(kInfBits), h = -__int_as_float(kInfBits);
    if (t < lanes * d) {
        const int a = t % d;
        for (int b = t / d; b < nb; b += lanes) {
            l = fminf(l, __ldcg(&part[(size_t)b * d + a]));
            h = fmaxf(h, __ldcg(&part[(size_t)(nb + b) * d + a]));
        }
    }
    __syncthreads();                              // sm's earlier contents are no longer read
    sm[t] = l;
    sm[blockDim.x + t] = h;
    __syncthreads();
    if (t < d) {
        for (int k = 1; k < lanes; k++) {
            l = fminf(l, sm[k * d + t]);
            h = fmaxf(h, sm[blockDim.x + k * d + t]);
        }
        mn[t] = (double)l;
        mx[t] = (double)h;
    }
}

// Block layout: blockDim.x = d * rows_per_pass, so thread t always sees attribute t % d.
__global__ void k_minmax(const float *__restrict__ raw, int64_t n, int d, float *part,
                         uint32_t *ticket, double *mn, double *mx, uint32_t *flags)
{
    extern __shared__ float sm[];                 // 2 * blockDim.x
    const int t = threadIdx.x;
    const int rows_per_pass = blockDim.x / d;
    const int j = t % d;
    const int r0 = t / d;
    float lo = __int_as_float(kInfBits), hi = -__int_as_float(kInfBits);
    bool bad = false;
    if (r0 < rows_per_pass) {
        for (int64_t r = (int64_t)blockIdx.x * rows_per_pass + r0; r < n;
             r += (int64_t)gridDim.x * rows_per_pass) {
            float v = raw[r * d + j];
            bad |= !isfinite(v);
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
    }
    if (bad) atomicOr(&flags[0], 1u);
    sm[t] = lo;
    sm[blockDim.x + t] = hi;
    __syncthreads();
    if (t < d) {
        for (int q = 1; q < rows_per_pass; q++) {
            lo = fminf(lo, sm[q * d + t]);
            hi = fmaxf(hi, sm[blockDim.x + q * d + t]);
        }
        part[(size_t)blockIdx.x * d + t] = lo;
        part[(size_t)(gridDim.x + blockIdx.x) * d + t] = hi;
    }
    // the last block to finish folds all partials
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (t == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    fold_partials(part, d, sm, mn, mx);
    if (t == 0) *ticket = 0;
}

// The same reduction for d % 4 == 0 with float4 loads: thread t reads attributes
// 4g .. 4g+3 (g = t mod d/4) of rows t / (d/4), + rows_per_pass, ..., four rows in flight;
// blockDim.x is a multiple of d/4.
__global__ void k_minmax4(const float4 *__restrict__ raw4, int64_t n, int d, float *part,
                          uint32_t *ticket, double *mn, double *mx, uint32_t *flags)
{
    extern __shared__ float sm[];                 // 8 * blockDim.x
    const int q = d / 4;
    const int t = threadIdx.x;
    const int rpp = blockDim.x / q;
    const int g = t % q, r0 = t / q;
    float lo[4], hi[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        lo[c] = __int_as_float(kInfBits);
        hi[c] = -__int_as_float(kInfBits);
    }
    bool bad = false;
    const int64_t rs = (int64_t)gridDim.x * rpp;
    for (int64_t r = (int64_t)blockIdx.x * rpp + r0; r < n; r += 4 * rs) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (r + u * rs < n) v[u] = raw4[(r + u * rs) * q + g];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (r + u * rs >= n) break;
            const float e[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
            for (int c = 0; c < 4; c++) {
                bad |= !isfinite(e[c]);
                lo[c] = fminf(lo[c], e[c]);
                hi[c] = fmaxf(hi[c], e[c]);
            }
        }
    }
    if (bad) atomicOr(&flags[0], 1u);
#pragma unroll
    for (int c = 0; c < 4; c++) {
        sm[4 * t + c] = lo[c];
        sm[4 * blockDim.x + 4 * t + c] = hi[c];
    }
    __syncthreads();
    for (int a = t; a < d; a += blockDim.x) {
        const int ga = a / 4, c = a % 4;
        float l = __int_as_float(kInfBits), h = -__int_as_float(kInfBits);
        for (int k = 0; k < rpp; k++) {
            l = fminf(l, sm[4 * (ga + k * q) + c]);
            h = fmaxf(h, sm[4 * blockDim.x + 4 * (ga + k * q) + c]);
        }
        part[(size_t)blockIdx.x * d + a] = l;
        part[(size_t)(gridDim.x + blockIdx.x) * d + a] = h;
    }
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (t == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    fold_partials(part, d, sm, mn, mx);
    if (t == 0) *ticket = 0;
}

template <bool kBf16>
__device__ __forceinline__ float to_storage(double v)
{
    return kBf16 ? __bfloat162float(__double2bfloat16(v)) : __double2float_rn(v);
}

// Per attribute: the minimum (float64 and float32, equal), inv = RN(1/range) or 0 for a
// constant attribute, and inv split into floats ih + il (il = RN(inv - ih)); ih = il = 0
// where inv lies outside [2^-60, 2^60] (the float-float steps below would lose exactness),
// which sends every value of the attribute to the float64 expression.
struct ScaleAttr {
    double mn, inv;
    float mnf, ih, il;
};

__device__ __forceinline__ ScaleAttr scale_attr(double mn, double mx)
{
    ScaleAttr r;
    const double range = __dsub_rn(mx, mn);
    r.mn = mn;
    r.inv = range > 0.0 ? __drcp_rn(range) : 0.0;
    r.mnf = (float)mn;                                  // exact: the minimum is a float
    const bool ff = r.inv >= 0x1p-60 && r.inv <= 0x1p60 && isfinite(r.mnf);
    r.ih = ff ? __double2float_rn(r.inv) : 0.0f;
    r.il = ff ? __double2float_rn(__dsub_rn(r.inv, (double)r.ih)) : 0.0f;
    return r;
}

// The attribute table in shared memory, one array per field (consecutive attributes fall
// in consecutive banks).
struct ScaleTable {
    double *mn, *inv;
    float *mnf, *ih, *il;
    __device__ ScaleTable(void *base, int d)
    {
        mn = static_cast<double *>(base);
        inv = mn + d;
        mnf = reinterpret_cast<float *>(inv + d);
        ih = mnf + d;
        il = ih + d;
    }
    __device__ void put(int a, const ScaleAttr &r)
    {
        mn[a] = r.mn;
        inv[a] = r.inv;
        mnf[a] = r.mnf;
        ih[a] = r.ih;
        il[a] = r.il;
    }
    __device__ ScaleAttr get(int a) const
    {
        ScaleAttr r;
        r.mn = mn[a];
        r.inv = inv[a];
        r.mnf = mnf[a];
        r.ih = ih[a];
        r.il = il[a];
        return r;
    }
};

constexpr size_t scale_table_bytes(int d) { return (size_t)d * (2 * sizeof(double) + 3 * sizeof(float)); }

// RN_T((double(x) - mn) * inv), T = float32 or bfloat16, for inv > 0.  x - mn is split
// exactly into s + e (TwoSum) and multiplied by ih + il in float-float (the FMA gives s*ih
// exactly as p + pe): z = zh + zl lies within 2^-44.8 |z| of the float64 product y (its two
// roundings, the split of inv, the dropped e*il and the roundings of the small terms).  If
// z is farther than 2^-16 of a half-spacing of T (2^-12 for bfloat16) from T's rounding
// midpoints, RN_T(y) is the T value nearest z; otherwise, and below 2^-90 where the FMA
// step may underflow, the float64 expression decides (about 0.1 % of values).
template <bool kBf16>
__device__ __forceinline__ float scaled_value(float x, const ScaleAttr &A)
{
    const float s = __fsub_rn(x, A.mnf);
    if (s == 0.0f) return 0.0f;                         // x == mn: y = +0
    const float bb = __fsub_rn(s, x);
    const float e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(-A.mnf, bb));
    const float p = __fmul_rn(s, A.ih);
    const float pe = __fmaf_rn(s, A.ih, -p);
    const float t = __fadd_rn(pe, __fadd_rn(__fmul_rn(s, A.il), __fmul_rn(e, A.ih)));
    const float zh = __fadd_rn(p, t);                   // Fast2Sum: |t| <= 2^-22 |p|
    const float zl = __fsub_rn(t, __fsub_rn(zh, p));
    if (zh >= 0x1p-90f && zh < 0x1p100f) {
        const uint32_t b = __float_as_uint(zh);
        if (!kBf16) {
            // half the spacing of floats around zh (the smaller one below a power of two)
            float hs = __uint_as_float(((b >> 23) - 24u) << 23);
            if ((b & 0x7FFFFFu) == 0) hs = __fmul_rn(hs, 0.5f);
            if (fabsf(zl) <= __fsub_rn(hs, __fmul_rn(hs, 0x1p-16f))) return zh;
        } else {
            const uint32_t cb = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;   // zh to 8 bits
            const float c = __uint_as_float(cb);
            const float u = __fadd_rn(__fsub_rn(zh, c), zl);                       // z - c
            float hs = __uint_as_float(((cb >> 23) - 8u) << 23);
            if ((cb & 0x7FFFFFu) == 0) hs = __fmul_rn(hs, 0.5f);
            if (fabsf(u) <= __fsub_rn(hs, __fmul_rn(hs, 0x1p-12f))) return c;
        }
    }
    return to_storage<kBf16>(__dmul_rn(__dsub_rn((double)x, A.mn), A.inv));
}

// bfloat16 points widened to float32 (exact).
__global__ void k_widen_bf16(const uint16_t *__restrict__ in, float *__restrict__ out, int64_t count)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = __uint_as_float((uint32_t)in[e] << 16);
}

// A thread keeps the attributes it scales in registers: the launch makes the grid stride
// (in elements) a multiple of d, so every element a thread visits has the same attribute
// (the same four for a float4); other strides look the attributes up per element.
template <bool kVec4, bool kBf16>
__global__ void k_scale_apply(const float *__restrict__ raw, float *__restrict__ x, int64_t n,
                              int d, const double *__restrict__ mn, const double *__restrict__ mx)
{
    extern __shared__ __align__(16) unsigned char sraw[];
    ScaleTable tab(sraw, d);
    for (int a = threadIdx.x; a < d; a += blockDim.x) tab.put(a, scale_attr(mn[a], mx[a]));
    __syncthreads();
    const int64_t total = n * d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (kVec4) {
        // four float4 per thread in flight; a float4 holds attributes a..a+3 of one row
        const int64_t total4 = total / 4;
        const float4 *r4 = reinterpret_cast<const float4 *>(raw);
        float4 *x4 = reinterpret_cast<float4 *>(x);
        const bool fixed = (4 * stride) % d == 0;
        const int a0 = (int)((4 * first) % d);
        ScaleAttr A[4];
#pragma unroll
        for (int c = 0; c < 4; c++) A[c] = tab.get(a0 + c);
        for (int64_t e0 = first; e0 < total4; e0 += 4 * stride) {
            float4 v[4];
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (e0 + q * stride < total4) v[q] = r4[e0 + q * stride];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int64_t e = e0 + q * stride;
                if (e >= total4) break;
                if (!fixed) {
                    const int a = (int)((e * 4) % d);
#pragma unroll
                    for (int c = 0; c < 4; c++) A[c] = tab.get(a + c);
                }
                float o[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
                for (int c = 0; c < 4; c++) o[c] = A[c].inv != 0.0 ? scaled_value<kBf16>(o[c], A[c]) : 0.0f;
                x4[e] = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
    } else {
        const bool fixed = stride % d == 0;
        ScaleAttr A = tab.get((int)(first % d));
        for (int64_t e = first; e < total; e += stride) {
            if (!fixed) A = tab.get((int)(e % d));
            x[e] = A.inv != 0.0 ? scaled_value<kBf16>(raw[e], A) : 0.0f;
        }
    }
}

// Independent sets (SegTable units): per unit, the column minima and maxima of its rows.
// With d <= blockDim.x, thread t reads attribute t % d of rows t / d, t / d + lanes, ...
__global__ void k_unit_minmax(const float *__restrict__ raw, SegTable t, int d, float *part, uint32_t *flags)
{
    extern __shared__ float sm[];                 // 2 * blockDim.x
    const int u = blockIdx.x;
    const int64_t row0 = t.seg_start[t.unit_seg[u]] + t.unit_start[u];
    const int rows = t.unit_count[u];
    const int lanes = d <= (int)blockDim.x ? (int)blockDim.x / d : 1;
    bool bad = false;
    for (int j0 = 0; j0 < d; j0 += (int)blockDim.x) {
        const int j = j0 + (d <= (int)blockDim.x ? (int)threadIdx.x % d : (int)threadIdx.x);
        const int r0 = d <= (int)blockDim.x ? (int)threadIdx.x / d : 0;
        float lo = __int_as_float(kInfBits), hi = -__int_as_float(kInfBits);
        if (j < d && r0 < lanes) {
            for (int r = r0; r < rows; r += lanes) {
                const float v = raw[(row0 + r) * d + j];
                bad |= !isfinite(v);
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
            }
        }
        sm[threadIdx.x] = lo;
        sm[blockDim.x + threadIdx.x] = hi;
        __syncthreads();
        if (j < d && r0 == 0) {
            for (int q = 1; q < lanes; q++) {
                lo = fminf(lo, sm[q * d + threadIdx.x]);
                hi = fmaxf(hi, sm[blockDim.x + q * d + threadIdx.x]);
            }
            part[(size_t)u * d + j] = lo;
            part[((size_t)t.n_units + u) * d + j] = hi;
        }
        __syncthreads();
    }
    if (bad) atomicOr(&flags[0], 1u);
}

// Per set: fold its units' partials (exact in any order) into mn / mx.
__global__ void k_seg_minmax_fold(const float *part, SegTable t, const int32_t *seg_unit0, int d, double *mn,
                                  double *mx)
{
    const int s = blockIdx.x;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        float lo = __int_as_float(kInfBits), hi = -__int_as_float(kInfBits);
        for (int u = seg_unit0[s]; u < seg_unit0[s + 1]; u++) {
            lo = fminf(lo, part[(size_t)u * d + j]);
            hi = fmaxf(hi, part[((size_t)t.n_units + u) * d + j]);
        }
        mn[(size_t)s * d + j] = (double)lo;
        mx[(size_t)s * d + j] = (double)hi;
    }
}

// Per unit: its rows scaled with its set's minimum and range, the same formula as above.
// With d <= blockDim.x thread t scales attribute t mod d of rows t / d, + blockDim.x / d, ...
// (its attribute in registers); wider points are scaled row by row.
__global__ void k_unit_scale(const float *__restrict__ raw, float *__restrict__ x, SegTable t, int d,
                             const double *__restrict__ mn, const double *__restrict__ mx)
{
    extern __shared__ __align__(16) unsigned char sraw[];
    ScaleTable tab(sraw, d);
    const int u = blockIdx.x;
    const int s = t.unit_seg[u];
    for (int a = threadIdx.x; a < d; a += blockDim.x) tab.put(a, scale_attr(mn[(size_t)s * d + a], mx[(size_t)s * d + a]));
    __syncthreads();
    const int64_t row0 = t.seg_start[s] + t.unit_start[u];
    const int rows = t.unit_count[u];
    if (d <= (int)blockDim.x) {
        const int per = (int)blockDim.x / d;
        if ((int)threadIdx.x >= per * d) return;
        const int a = (int)threadIdx.x % d;
        const ScaleAttr A = tab.get(a);
        for (int r = (int)threadIdx.x / d; r < rows; r += per) {
            const int64_t e = (row0 + r) * d + a;
            x[e] = A.inv != 0.0 ? scaled_value<false>(raw[e], A) : 0.0f;
        }
    } else {
        for (int r = 0; r < rows; r++)
            for (int a = threadIdx.x; a < d; a += blockDim.x) {
                const int64_t e = (row0 + r) * d + a;
                const ScaleAttr A = tab.get(a);
                x[e] = A.inv != 0.0 ? scaled_value<false>(raw[e], A) : 0.0f;
            }
    }
}

}  // namespace

cudaError_t launch_seg_scale(const float *raw, float *x, const SegTable &t, const int32_t *seg_unit0, int d,
                             float *part, double *mn, double *mx, uint32_t *flags, cudaStream_t st, KTimer *kt)
{
    const int thr = d < 256 ? ((d + 31) / 32) * 32 : 256;
    kt->begin(st);
    k_unit_minmax<<<t.n_units, 256, 2 * 256 * sizeof(float), st>>>(raw, t, d, part, flags);
    k_seg_minmax_fold<<<t.n_seg, thr, 0, st>>>(part, t, seg_unit0, d, mn, mx);
    kt->end(PSCL_K_SCALE_MINMAX, st);
    kt->begin(st);
    k_unit_scale<<<t.n_units, 256, scale_table_bytes(d), st>>>(raw, x, t, d, mn, mx);
    kt->end(PSCL_K_SCALE_APPLY, st);
    return cudaGetLastError();
}

namespace {
// at most sm_count * 4 blocks: the partials buffer (scale_part_floats) holds that many
void minmax_enqueue(const float *x, int64_t n, int d, float *part, uint32_t *ticket, double *mn, double *mx,
                    uint32_t *flags, int sm_count, cudaStream_t st)
{
    const bool vec = d % 4 == 0 && reinterpret_cast<uintptr_t>(x) % 16 == 0;
    const int threads = vec ? (d / 4) * (512 / (d / 4)) : d * (1024 / d);
    const int64_t rows_per_pass = vec ? threads / (d / 4) : threads / d;
    const int64_t want = (n + rows_per_pass - 1) / rows_per_pass;
    int grid = (int)(want < (int64_t)sm_count * 4 ? want : (int64_t)sm_count * 4);
    if (grid < 1) grid = 1;
    if (vec)
        k_minmax4<<<grid, threads, 8 * threads * sizeof(float), st>>>(reinterpret_cast<const float4 *>(x), n, d,
                                                                      part, ticket, mn, mx, flags);
    else
        k_minmax<<<grid, threads, 2 * threads * sizeof(float), st>>>(x, n, d, part, ticket, mn, mx, flags);
}
}  // namespace

cudaError_t launch_minmax(const float *x, int64_t n, int d, float *part, uint32_t *ticket, double *mn, double *mx,
                          uint32_t *flags, int sm_count, cudaStream_t st, KTimer *kt)
{
    kt->begin(st);
    minmax_enqueue(x, n, d, part, ticket, mn, mx, flags, sm_count, st);
    kt->end(PSCL_K_SCALE_MINMAX, st);
    return cudaGetLastError();
}

cudaError_t launch_widen_bf16(const uint16_t *in, float *out, int64_t count, int sm_count, cudaStream_t st)
{
    int64_t g = (count + 255) / 256;
    if (g > (int64_t)sm_count * 16) g = (int64_t)sm_count * 16;
    if (g < 1) g = 1;
    k_widen_bf16<<<(int)g, 256, 0, st>>>(in, out, count);
    return cudaGetLastError();
}

cudaError_t launch_scale(const float *raw, float *x, int64_t n, int d, float *part,
                         uint32_t *ticket, double *mn, double *mx, uint32_t *flags, int sm_count,
                         cudaStream_t st, KTimer *kt, int bf16)
{
    kt->begin(st);
    minmax_enqueue(raw, n, d, part, ticket, mn, mx, flags, sm_count, st);
    kt->end(PSCL_K_SCALE_MINMAX, st);
    bool vec = (d % 4) == 0;
    int64_t work = vec ? n * d / 4 : n * d;
    int64_t g2 = (work + 255) / 256;
    if (g2 > (int64_t)sm_count * 16) g2 = (int64_t)sm_count * 16;
    // a grid stride (256 g2 threads, 4 elements each when vectorised) that d divides keeps
    // each thread on the same attributes
    const int64_t per_block = vec ? 1024 : 256;
    const int64_t m = d / std::gcd(per_block, (int64_t)d);
    g2 = std::max<int64_t>(m, g2 - g2 % m);
    size_t smem = scale_table_bytes(d);
    kt->begin(st);
    if (vec && bf16)
        k_scale_apply<true, true><<<(int)g2, 256, smem, st>>>(raw, x, n, d, mn, mx);
    else if (vec)
        k_scale_apply<true, false><<<(int)g2, 256, smem, st>>>(raw, x, n, d, mn, mx);
    else if (bf16)
        k_scale_apply<false, true><<<(int)g2, 256, smem, st>>>(raw, x, n, d, mn, mx);
    else
        k_scale_apply<false, false><<<(int)g2, 256, smem, st>>>(raw, x, n, d, mn, mx);
    kt->end(PSCL_K_SCALE_APPLY, st);
    return cudaGetLastError();
}

size_t scale_part_floats(int64_t n, int d, int sm_count)
{
    (void)n;
    (void)d;
    return 2 * (size_t)sm_count * 4 * (size_t)d;
}

}  // namespace pscl
