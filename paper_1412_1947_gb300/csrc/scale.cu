// Feature scaling (Algorithm 1, step 1): min-max of every attribute to [0, 1].
//
//   mn_j = min_i x_ij, mx_j = max_i x_ij              (exact in any order)
//   x'_ij = RN( (double(x_ij) - mn_j) * (1 / (mx_j - mn_j)) )  in double, 0 if mx_j = mn_j,
//           rounded once to the storage type (float32, or bfloat16 kept in a float)
//
// Two kernels: a column min/max reduction (per-block partials, the last block to finish
// folds them) and an element-wise pass.  Both are HBM-bound: 2 reads + 1 write of n*d*4
// bytes in total.
#include <cuda_bf16.h>

#include "pscl_internal.cuh"

namespace pscl {
namespace {

constexpr uint32_t kInfBits = 0x7f800000u;

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
    for (int a = t; a < d; a += blockDim.x) {
        float l = __int_as_float(kInfBits), h = -__int_as_float(kInfBits);
        for (unsigned b = 0; b < gridDim.x; b++) {
            l = fminf(l, __ldcg(&part[(size_t)b * d + a]));
            h = fmaxf(h, __ldcg(&part[(size_t)(gridDim.x + b) * d + a]));
        }
        mn[a] = (double)l;
        mx[a] = (double)h;
    }
    if (t == 0) *ticket = 0;
}

template <bool kBf16>
__device__ __forceinline__ float to_storage(double v)
{
    return kBf16 ? __bfloat162float(__double2bfloat16(v)) : __double2float_rn(v);
}

// bfloat16 points widened to float32 (exact).
__global__ void k_widen_bf16(const uint16_t *__restrict__ in, float *__restrict__ out, int64_t count)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = __uint_as_float((uint32_t)in[e] << 16);
}

template <bool kVec4, bool kBf16>
__global__ void k_scale_apply(const float *__restrict__ raw, float *__restrict__ x, int64_t n,
                              int d, const double *__restrict__ mn, const double *__restrict__ mx)
{
    extern __shared__ double sd[];                // mn[d], inv[d]
    double *smn = sd, *sinv = sd + d;
    for (int a = threadIdx.x; a < d; a += blockDim.x) {
        double range = __dsub_rn(mx[a], mn[a]);
        smn[a] = mn[a];
        sinv[a] = range > 0.0 ? __drcp_rn(range) : 0.0;   // inv = 0 marks a constant attribute
    }
    __syncthreads();
    const int64_t total = n * d;
    if (kVec4) {
        const int64_t total4 = total / 4;
        const float4 *r4 = reinterpret_cast<const float4 *>(raw);
        float4 *x4 = reinterpret_cast<float4 *>(x);
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total4;
             e += (int64_t)gridDim.x * blockDim.x) {
            float4 v = r4[e];
            int a = (int)((e * 4) % d);
            float o[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                double inv = sinv[a + q];
                o[q] = inv != 0.0 ? to_storage<kBf16>(__dmul_rn(__dsub_rn((double)o[q], smn[a + q]), inv))
                                  : 0.0f;
            }
            x4[e] = make_float4(o[0], o[1], o[2], o[3]);
        }
    } else {
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
             e += (int64_t)gridDim.x * blockDim.x) {
            int a = (int)(e % d);
            double inv = sinv[a];
            x[e] = inv != 0.0 ? to_storage<kBf16>(__dmul_rn(__dsub_rn((double)raw[e], smn[a]), inv))
                              : 0.0f;
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
__global__ void k_unit_scale(const float *__restrict__ raw, float *__restrict__ x, SegTable t, int d,
                             const double *__restrict__ mn, const double *__restrict__ mx)
{
    const int u = blockIdx.x;
    const int s = t.unit_seg[u];
    const int64_t row0 = t.seg_start[s] + t.unit_start[u];
    const int64_t e0 = row0 * d, e1 = (row0 + t.unit_count[u]) * d;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int a = (int)((e - e0) % d);
        const double lo = mn[(size_t)s * d + a];
        const double range = __dsub_rn(mx[(size_t)s * d + a], lo);
        x[e] = range > 0.0 ? __double2float_rn(__dmul_rn(__dsub_rn((double)raw[e], lo), __drcp_rn(range))) : 0.0f;
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
    k_unit_scale<<<t.n_units, 256, 0, st>>>(raw, x, t, d, mn, mx);
    kt->end(PSCL_K_SCALE_APPLY, st);
    return cudaGetLastError();
}

cudaError_t launch_minmax(const float *x, int64_t n, int d, float *part, uint32_t *ticket, double *mn, double *mx,
                          uint32_t *flags, int sm_count, cudaStream_t st, KTimer *kt)
{
    int threads = d * (1024 / d);
    int64_t rows_per_pass = threads / d;
    int64_t want = (n + rows_per_pass - 1) / rows_per_pass;
    int grid = (int)(want < (int64_t)sm_count * 4 ? want : (int64_t)sm_count * 4);
    if (grid < 1) grid = 1;
    kt->begin(st);
    k_minmax<<<grid, threads, 2 * threads * sizeof(float), st>>>(x, n, d, part, ticket, mn, mx, flags);
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
    int threads = d * (1024 / d);
    int64_t rows_per_pass = threads / d;
    int64_t want = (n + rows_per_pass - 1) / rows_per_pass;
    int grid = (int)(want < (int64_t)sm_count * 4 ? want : (int64_t)sm_count * 4);
    if (grid < 1) grid = 1;
    kt->begin(st);
    k_minmax<<<grid, threads, 2 * threads * sizeof(float), st>>>(raw, n, d, part, ticket, mn, mx, flags);
    kt->end(PSCL_K_SCALE_MINMAX, st);
    bool vec = (d % 4) == 0;
    int64_t work = vec ? n * d / 4 : n * d;
    int64_t g2 = (work + 255) / 256;
    if (g2 > (int64_t)sm_count * 16) g2 = (int64_t)sm_count * 16;
    if (g2 < 1) g2 = 1;
    size_t smem = 2 * (size_t)d * sizeof(double);
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
