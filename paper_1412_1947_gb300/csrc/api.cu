// C ABI of the pscl library: contexts, jobs, planning and the order of launches.
// The kernels live in scale.cu, peel.cu and lloyd.cu; this file only allocates,
// uploads the small index tables, queues launches and copies results out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pscl_internal.cuh"

using namespace pscl;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

void pscl::set_last_error(const char *msg) { g_err = msg; }

#define CU(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError(); /* clear a non-sticky error so later calls start clean */   \
            return fail(PSCL_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                \
        }                                                                                   \
    } while (0)

// ------------------------------------------------------------------ objects
struct pscl_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    size_t in_use = 0;
    int sm_count = 0;
};

struct Alloc {
    void *p;
    size_t bytes;
};

// Anything that owns device allocations charged to a context's budget.
struct Owner {
    pscl_ctx *ctx = nullptr;
    std::vector<Alloc> allocs;
};

// One Lloyd launch plan: tables on the device and their host copies.
struct LloydPlan {
    int n_seg = 0, n_units = 0, kmax = 0, d = 0, max_unit = 0;
    int64_t rows = 0, P = 0;
    std::vector<int64_t> seg_start;
    std::vector<int32_t> seg_size, cen_off, k_eff, unit_seg, unit_start, unit_count, seg_unit0;
    int64_t *d_seg_start = nullptr;
    int32_t *d_i32 = nullptr;       // seg_size | cen_off | k_eff | unit_seg | unit_start | unit_count | seg_unit0
    const int32_t *d_unit0() const { return d_i32 + 3 * n_seg + 3 * n_units; }
    int32_t *d_split = nullptr;     // CTA splits of the units for 1..4 CTAs per SM
    int split_off[5] = {};
    SegTable table() const
    {
        SegTable t;
        t.seg_start = d_seg_start;
        t.seg_size = d_i32;
        t.cen_off = d_i32 + n_seg;
        t.k_eff = d_i32 + 2 * n_seg;
        t.unit_seg = d_i32 + 3 * n_seg;
        t.unit_start = d_i32 + 3 * n_seg + n_units;
        t.unit_count = d_i32 + 3 * n_seg + 2 * n_units;
        t.n_seg = n_seg;
        t.n_units = n_units;
        t.split = d_split;
        for (int m = 0; m < 5; m++) t.split_off[m] = split_off[m];
        return t;
    }
};

struct pscl_job : Owner {
    int64_t n = 0;
    int d = 0;
    int state = 0;                    // 0 loaded, 1 scaled, 2 subclustered, 3 clustered
    // options
    int plain = 0, trace = 0, first_k = 0, graph = 0, ktiming = 0, rpt = 0, pool_w = 0;
    int peel_rounds = 0;              // rounds per distance pass of the peel (0: default)
    uint32_t wait_limit = 0;          // polls of a bounded device-side wait (0: default)
    int test_stall = 0;               // test hook: a wait that cannot complete (1 peel, 2 tensor core)
    int peel_grid = 0;                // most CTAs of the peel's launch (0: as many as fit)
    KTimer kt;                        // launch counts (+ events when timing) of the last run
    // input and scaling
    int dtype = PSCL_F32;
    const float *dev_in = nullptr;    // caller's device buffer, or raw (float32 points)
    float *raw = nullptr;             // owned copy of host input, or the widened bfloat16 input
    const uint16_t *in16 = nullptr;   // bfloat16 input: the caller's device buffer, or raw16
    uint16_t *raw16 = nullptr;        // owned copy of bfloat16 host input
    float *x = nullptr;               // scaled points (original order)
    double *mn = nullptr, *mx = nullptr;
    float *part = nullptr;
    uint32_t *tickets = nullptr;      // [0] scale, [1] sse
    PeelCtl *ctl = nullptr;
    uint32_t *flags = nullptr;        // kFlagWords
    // subcluster plan
    int64_t N = 0;
    int local_k = 0, iters = 0, prec = 0;
    uint64_t seed = 0;
    int64_t S = 0, P = 0;
    std::vector<int64_t> seg_off;
    PeelBuffers pb{};
    bool peel_alloc = false;
    LloydPlan lp;
    float *cl = nullptr;              // P x d local centers
    unsigned long long *acc_l = nullptr;
    int32_t *cnt_l = nullptr;         // 2P
    int32_t *lab_l = nullptr;         // n (packed order)
    int32_t *trace_l = nullptr;       // iters x n
    int64_t trace_l_len = 0;
    // final plan
    int final_k = 0, fiters = 0, fprec = 0;
    uint64_t fseed = 0;
    LloydPlan fp;
    // the SSE pass's row tables: all n rows as one set of 256 centers (final_k > 256) and of
    // the remaining final_k mod 256 centers (final_k itself when it is at most 256)
    LloydPlan sp256, sprem;
    // the final Lloyd's row tables for the same chunked search (final_k > 256 only)
    LloydPlan fp256, fprem;
    float *cf = nullptr;
    unsigned long long *acc_f = nullptr;
    int32_t *cnt_f = nullptr;
    int32_t *lab_f = nullptr;         // P
    int32_t *trace_f = nullptr;
    int64_t trace_f_len = 0;
    int32_t *labels = nullptr;        // n
    double *blk_sse = nullptr;
    double *sse = nullptr;
    int sse_blocks = 0;
    // phases
    cudaEvent_t ev[6] = {};
    bool ev_ok = false;
    // recorded pipeline
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey[8] = {};
    // Algorithm 2 (unequal-sized subclustering): m landmarks and the grouping's buffers
    int unequal_m = 0;
    float *u_lm = nullptr;
    int32_t *u_group = nullptr;
    uint32_t *u_cnt = nullptr, *u_total = nullptr;
    double *u_lo = nullptr, *u_hi = nullptr;
    // serving: the peel goes to a stream shared by all jobs (cooperative launches one at a time)
    cudaStream_t coop = nullptr;
    cudaEvent_t coop_ev[2] = {};
};

// ------------------------------------------------------------------ memory
static int job_alloc(Owner *j, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    pscl_ctx *c = j->ctx;
    if (c->budget && c->in_use + bytes > c->budget)
        return fail(PSCL_ENOMEM, "device-memory budget exceeded: %zu in use + %zu requested > %zu",
                    c->in_use, bytes, c->budget);
    // stream-ordered: neither allocating nor freeing waits for other streams' work
    cudaError_t e = cudaMallocAsync(p, bytes, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? PSCL_ENOMEM : PSCL_ECUDA,
                    "cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    j->allocs.push_back({*p, bytes});
    c->in_use += bytes;
    return PSCL_OK;
}

static void job_free(Owner *j, void *p)
{
    if (!p) return;
    for (size_t i = 0; i < j->allocs.size(); i++) {
        if (j->allocs[i].p == p) {
            cudaFreeAsync(p, j->ctx->stream);
            j->ctx->in_use -= j->allocs[i].bytes;
            j->allocs.erase(j->allocs.begin() + i);
            return;
        }
    }
}

template <class T>
static int A(Owner *j, T **p, size_t count)
{
    void *v = nullptr;
    int rc = job_alloc(j, &v, count * sizeof(T));
    *p = static_cast<T *>(v);
    return rc;
}

#define TRY(x)                    \
    do {                          \
        int rc_ = (x);            \
        if (rc_ != PSCL_OK) return rc_; \
    } while (0)

static void drop_graph(pscl_job *j)
{
    if (j->gexec) {
        cudaGraphExecDestroy(j->gexec);
        j->gexec = nullptr;
    }
}

// ------------------------------------------------------------------ context
extern "C" int pscl_ctx_create(pscl_ctx **out, int device, size_t budget, void *stream)
{
    if (!out) return fail(PSCL_EINVAL, "out is NULL");
    int ndev = 0;
    CU(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(PSCL_EINVAL, "device %d out of range (%d devices)", device, ndev);
    CU(cudaSetDevice(device));
    pscl_ctx *c = new pscl_ctx();
    c->device = device;
    c->budget = budget;
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        c->sm_count < 1) {
        delete c;
        cudaGetLastError();
        return fail(PSCL_ECUDA, "device %d: no multiprocessor count", device);
    }
    {   // keep freed pool memory for the next job instead of returning it at every sync
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    }
    if (stream) {
        c->stream = static_cast<cudaStream_t>(stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return fail(PSCL_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    *out = c;
    g_err.clear();
    return PSCL_OK;
}

extern "C" int pscl_ctx_destroy(pscl_ctx *c)
{
    if (!c) return fail(PSCL_EINVAL, "ctx is NULL");
    cudaSetDevice(c->device);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return PSCL_OK;
}

extern "C" size_t pscl_ctx_bytes_in_use(const pscl_ctx *c) { return c ? c->in_use : 0; }

extern "C" const char *pscl_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ jobs
static int load_points(pscl_job *j, const void *points, int on_device)
{
    if (!points) return fail(PSCL_EINVAL, "points is NULL");
    if (j->dtype == PSCL_BF16) {
        // bfloat16 points: widened to float32 at the start of every run (enqueue_scale)
        if (!j->raw) TRY(A(j, &j->raw, (size_t)j->n * j->d));
        if (on_device) {
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, points) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
                at.device != j->ctx->device) {
                cudaGetLastError();
                return fail(PSCL_EINVAL, "points_on_device=1 but the pointer is not device memory of device %d",
                            j->ctx->device);
            }
            j->in16 = static_cast<const uint16_t *>(points);
        } else {
            if (!j->raw16) TRY(A(j, &j->raw16, (size_t)j->n * j->d));
            CU(cudaMemcpyAsync(j->raw16, points, (size_t)j->n * j->d * sizeof(uint16_t), cudaMemcpyHostToDevice,
                               j->ctx->stream));
            j->in16 = j->raw16;
        }
        j->dev_in = j->raw;
        j->state = 0;
        return PSCL_OK;
    }
    if (on_device) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, points) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
            at.device != j->ctx->device) {
            cudaGetLastError();
            return fail(PSCL_EINVAL, "points_on_device=1 but the pointer is not device memory of device %d",
                        j->ctx->device);
        }
        if (((uintptr_t)points & 15) != 0) return fail(PSCL_EINVAL, "device points must be 16-byte aligned");
        j->dev_in = static_cast<const float *>(points);
    } else {
        if (!j->raw) TRY(A(j, &j->raw, (size_t)j->n * j->d));
        CU(cudaMemcpyAsync(j->raw, points, (size_t)j->n * j->d * sizeof(float), cudaMemcpyHostToDevice,
                           j->ctx->stream));
        j->dev_in = j->raw;
    }
    j->state = 0;
    return PSCL_OK;
}

extern "C" int pscl_job_create(pscl_ctx *c, const void *points, int dtype, int64_t n, int32_t d,
                               int on_device, pscl_job **out)
{
    if (!c || !out) return fail(PSCL_EINVAL, "ctx or out is NULL");
    if (dtype != PSCL_F32 && dtype != PSCL_BF16) return fail(PSCL_EINVAL, "dtype %d is not PSCL_F32 or PSCL_BF16", dtype);
    if (n < 1 || n > (int64_t)INT32_MAX) return fail(PSCL_EINVAL, "n=%lld outside 1..2^31-1", (long long)n);
    if (d < 1 || d > kMaxD) return fail(PSCL_EINVAL, "d=%d outside 1..%d", d, kMaxD);
    CU(cudaSetDevice(c->device));
    pscl_job *j = new pscl_job();
    j->ctx = c;
    j->n = n;
    j->d = d;
    j->dtype = dtype;
    int rc = PSCL_OK;
    if (!rc) rc = A(j, &j->x, (size_t)n * d);
    if (!rc) rc = A(j, &j->mn, d);
    if (!rc) rc = A(j, &j->mx, d);
    if (!rc) rc = A(j, &j->part, scale_part_floats(n, d, c->sm_count));
    if (!rc) rc = A(j, &j->tickets, 8);
    if (!rc) rc = A(j, &j->ctl, 1);
    if (!rc) rc = A(j, &j->flags, kFlagWords);
    if (!rc && cudaMemsetAsync(j->tickets, 0, 8 * sizeof(uint32_t), c->stream) != cudaSuccess) rc = PSCL_ECUDA;
    if (!rc && cudaMemsetAsync(j->flags, 0, kFlagWords * sizeof(uint32_t), c->stream) != cudaSuccess) rc = PSCL_ECUDA;
    if (!rc) rc = load_points(j, points, on_device);
    if (!rc) {
        for (int i = 0; i < 6 && !rc; i++)
            if (cudaEventCreate(&j->ev[i]) != cudaSuccess) rc = PSCL_ECUDA;
    }
    if (rc) {
        std::string msg = g_err;
        pscl_job_destroy(j);
        g_err = msg;
        return rc;
    }
    *out = j;
    return PSCL_OK;
}

extern "C" int pscl_job_load(pscl_job *j, const void *points, int on_device)
{
    if (!j) return fail(PSCL_EINVAL, "job is NULL");
    CU(cudaSetDevice(j->ctx->device));
    return load_points(j, points, on_device);
}

extern "C" int pscl_job_set_option(pscl_job *j, int opt, int64_t v)
{
    if (!j) return fail(PSCL_EINVAL, "job is NULL");
    switch (opt) {
    case PSCL_OPT_PLAIN_LLOYD: j->plain = v != 0; break;
    case PSCL_OPT_TRACE_LABELS: j->trace = v != 0; break;
    case PSCL_OPT_INIT_FIRST_K: j->first_k = v != 0; break;
    case PSCL_OPT_GRAPH: j->graph = v != 0; break;
    case PSCL_OPT_KERNEL_TIMING: j->ktiming = v != 0; break;
    case PSCL_OPT_ROWS_PER_THREAD:
        if (v < 0 || v > 2) return fail(PSCL_EINVAL, "rows per thread must be 0, 1 or 2");
        j->rpt = (int)v;
        break;
    case PSCL_OPT_PEEL_ROUNDS:
        if (v < 0 || v > kMaxEpoch) return fail(PSCL_EINVAL, "peel rounds per pass must be 0..%d", kMaxEpoch);
        j->peel_rounds = (int)v;
        break;
    case PSCL_OPT_WAIT_LIMIT:
        if (v < 0 || v > 0xFFFFFFFFll) return fail(PSCL_EINVAL, "wait limit must be 0..2^32-1");
        j->wait_limit = (uint32_t)v;
        break;
    case PSCL_OPT_TEST_STALL:
        if (v < 0 || v > 2) return fail(PSCL_EINVAL, "test stall must be 0, 1 or 2");
        j->test_stall = (int)v;
        break;
    case PSCL_OPT_PEEL_GRID:
        if (v < 0 || v > (1 << 20)) return fail(PSCL_EINVAL, "peel grid must be 0..2^20");
        j->peel_grid = (int)v;
        drop_graph(j);
        break;
    case PSCL_OPT_POOL_WEIGHTED:
        // the weights sum to n in an int32 count, and w x to at most n 2^32 in 64 bits
        if (v != 0 && j->n >= ((int64_t)1 << 31)) return fail(PSCL_EINVAL, "weighted pooling needs n < 2^31");
        j->pool_w = v != 0;
        break;
    default: return fail(PSCL_EINVAL, "unknown option %d", opt);
    }
    drop_graph(j);
    return PSCL_OK;
}

extern "C" int pscl_job_destroy(pscl_job *j)
{
    if (!j) return fail(PSCL_EINVAL, "job is NULL");
    cudaSetDevice(j->ctx->device);
    cudaStreamSynchronize(j->ctx->stream);
    drop_graph(j);
    for (auto &a : j->allocs) {
        cudaFreeAsync(a.p, j->ctx->stream);
        j->ctx->in_use -= a.bytes;
    }
    for (int i = 0; i < 6; i++)
        if (j->ev[i]) cudaEventDestroy(j->ev[i]);
    for (int i = 0; i < 2; i++)
        if (j->coop_ev[i]) cudaEventDestroy(j->coop_ev[i]);
    if (j->kt.ev) {
        for (int i = 0; i < 2 * j->kt.cap; i++) cudaEventDestroy(j->kt.ev[i]);
        delete[] j->kt.ev;
        delete[] j->kt.tag;
    }
    delete j;
    return PSCL_OK;
}

// ------------------------------------------------------------------ planning
static int64_t unit_target(int64_t rows, int sm_count, int64_t unit_rows)
{
    const int64_t target = unit_rows > 0 ? unit_rows : rows / ((int64_t)sm_count * 4);
    return std::max<int64_t>(unit_rows > 0 ? 32 : 128, std::min<int64_t>(1024, target));
}

// rows per unit of a set of m rows (a multiple of 32)
static int64_t unit_size(int64_t m, int64_t target)
{
    const int64_t nu = (m + target - 1) / target;
    return ((m + nu - 1) / nu + 31) / 32 * 32;
}

// Work units: every set is cut into ceil(m / target) near-equal pieces (multiples of 32
// rows), target chosen so that a launch has a few units per SM (or given: unit_rows, at
// most 1024 rows, the shared-accumulator bound of the assignment kernel).
static int build_lloyd_plan(Owner *j, LloydPlan &p, const std::vector<int64_t> &starts,
                            const std::vector<int32_t> &sizes, const std::vector<int32_t> &keff,
                            int64_t unit_rows = 0)
{
    p.n_seg = (int)sizes.size();
    p.seg_start = starts;
    p.seg_size = sizes;
    p.k_eff = keff;
    p.cen_off.assign(p.n_seg, 0);
    p.kmax = 0;
    int64_t P = 0, rows = 0;
    for (int s = 0; s < p.n_seg; s++) {
        p.cen_off[s] = (int32_t)P;
        P += keff[s];
        rows += sizes[s];
        p.kmax = std::max(p.kmax, keff[s]);
    }
    p.P = P;
    p.rows = rows;
    const int64_t target = unit_target(rows, j->ctx->sm_count, unit_rows);
    p.unit_seg.clear();
    p.unit_start.clear();
    p.unit_count.clear();
    p.seg_unit0.assign(p.n_seg + 1, 0);
    for (int s = 0; s < p.n_seg; s++) {
        p.seg_unit0[s] = (int32_t)p.unit_seg.size();
        const int64_t m = sizes[s];
        const int64_t us = unit_size(m, target);
        for (int64_t r = 0; r < m; r += us) {
            p.unit_seg.push_back(s);
            p.unit_start.push_back((int32_t)r);
            p.unit_count.push_back((int32_t)std::min<int64_t>(us, m - r));
        }
    }
    p.n_units = (int)p.unit_seg.size();
    p.seg_unit0[p.n_seg] = p.n_units;
    p.max_unit = p.unit_count.empty() ? 0 : *std::max_element(p.unit_count.begin(), p.unit_count.end());
    job_free(j, p.d_seg_start);
    job_free(j, p.d_i32);
    p.d_seg_start = nullptr;
    p.d_i32 = nullptr;
    TRY(A(j, &p.d_seg_start, p.n_seg));
    TRY(A(j, &p.d_i32, 4 * (size_t)p.n_seg + 3 * (size_t)p.n_units + 1));
    std::vector<int32_t> packed;
    packed.reserve(4 * p.n_seg + 3 * p.n_units + 1);
    packed.insert(packed.end(), p.seg_size.begin(), p.seg_size.end());
    packed.insert(packed.end(), p.cen_off.begin(), p.cen_off.end());
    packed.insert(packed.end(), p.k_eff.begin(), p.k_eff.end());
    packed.insert(packed.end(), p.unit_seg.begin(), p.unit_seg.end());
    packed.insert(packed.end(), p.unit_start.begin(), p.unit_start.end());
    packed.insert(packed.end(), p.unit_count.begin(), p.unit_count.end());
    packed.insert(packed.end(), p.seg_unit0.begin(), p.seg_unit0.end());
    cudaStream_t st = j->ctx->stream;
    CU(cudaMemcpyAsync(p.d_seg_start, p.seg_start.data(), p.n_seg * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(p.d_i32, packed.data(), packed.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    // Contiguous unit ranges of near-equal weight for persistent launches of G = m * SMs
    // CTAs (rows, plus a set-up allowance wherever a range has to start a new set).
    const int sm = j->ctx->sm_count;
    std::vector<int64_t> wpre(p.n_units + 1, 0);
    for (int u = 0; u < p.n_units; u++) {
        const bool first = u == 0 || p.unit_seg[u] != p.unit_seg[u - 1];
        wpre[u + 1] = wpre[u] + p.unit_count[u] + (first ? 256 : 0);
    }
    std::vector<int32_t> split;
    for (int m = 1; m <= 4; m++) {
        const int G = m * sm;
        p.split_off[m] = (int)split.size();
        int u = 0;
        for (int c = 0; c <= G; c++) {
            const int64_t target = wpre[p.n_units] * c / G;
            while (u < p.n_units && wpre[u] < target) u++;
            split.push_back(c == G ? p.n_units : u);
        }
    }
    job_free(j, p.d_split);
    p.d_split = nullptr;
    TRY(A(j, &p.d_split, split.size()));
    CU(cudaMemcpyAsync(p.d_split, split.data(), split.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    // (pageable sources: cudaMemcpyAsync returns once it has staged them)
    return PSCL_OK;
}

static int check_prec(int prec)
{
    if (prec < PSCL_PREC_FP32 || prec > PSCL_PREC_TC)
        return fail(PSCL_EINVAL, "unknown precision %d", prec);
    return PSCL_OK;
}

static int alloc_subcluster_buffers(pscl_job *j);
static int plan_local(pscl_job *j, const std::vector<int64_t> &starts, const std::vector<int32_t> &sizes,
                      int32_t local_k);
static int plan_trace(pscl_job *j, int32_t iters);

static int plan_subcluster(pscl_job *j, int64_t N, int32_t local_k, int32_t iters, uint64_t seed, int prec)
{
    if (N < 1) return fail(PSCL_EINVAL, "N=%lld < 1", (long long)N);
    if (local_k < 1 || local_k > kMaxK) return fail(PSCL_EINVAL, "local_k=%d outside 1..%d", local_k, kMaxK);
    if (iters < 0) return fail(PSCL_EINVAL, "iters < 0");
    TRY(check_prec(prec));
    TRY(alloc_subcluster_buffers(j));
    const int64_t n = j->n;
    const int d = j->d;
    const bool same = N == j->N && local_k == j->local_k;
    j->iters = iters;
    j->seed = seed;
    j->prec = prec;
    if (!same) {
        drop_graph(j);
        j->N = N;
        j->local_k = local_k;
        const int64_t S = (n + N - 1) / N;
        std::vector<int64_t> starts(S);
        std::vector<int32_t> sizes(S);
        for (int64_t s = 0; s < S; s++) {
            starts[s] = s * N;
            sizes[s] = (int32_t)std::min<int64_t>(N, n - s * N);
        }
        job_free(j, j->pb.landmarks);
        j->pb.landmarks = nullptr;
        TRY(A(j, &j->pb.landmarks, (size_t)S * d));
        TRY(plan_local(j, starts, sizes, local_k));
    }
    return plan_trace(j, iters);
}

// The subcluster buffers every scheme uses (allocated once per job).
static int alloc_subcluster_buffers(pscl_job *j)
{
    const int64_t n = j->n;
    const int d = j->d;
    if (!j->peel_alloc) {
        PeelBuffers &b = j->pb;
        b.x = j->x;
        b.ord_ld = (n + 3) & ~(int64_t)3;
        b.nbuckets = peel_buckets(n);
        TRY(A(j, &b.rnd, n));
        TRY(A(j, &b.pflag, 2 * (size_t)n));
        TRY(A(j, &b.ord, (size_t)d * b.ord_ld));
        TRY(A(j, &b.bcnt, (size_t)d * b.nbuckets));
        TRY(A(j, &b.bcs, (size_t)d * b.nbuckets));
        TRY(A(j, &b.lidx, 2 * (size_t)n));
        TRY(A(j, &b.kpos, 2 * (size_t)n));
        TRY(A(j, &b.band_k32, n));
        TRY(A(j, &b.band_pos, n));
        TRY(A(j, &b.gkey, n));
        TRY(A(j, &b.gpos, n));
        TRY(A(j, &b.akey, n));
        TRY(A(j, &b.apos, n));
        TRY(A(j, &b.pcnt, 256 * (size_t)perm_grid(n, j->ctx->sm_count)));
        TRY(A(j, &b.perm, n));
        TRY(A(j, &b.xseg, (size_t)n * d));
        TRY(A(j, &j->lab_l, n));
        b.ctl = j->ctl;
        b.flags = j->flags;
        j->peel_alloc = true;
    }
    return PSCL_OK;
}

// The local Lloyd plan over the subclusters (starts, sizes), their centers and sums.
static int plan_local(pscl_job *j, const std::vector<int64_t> &starts, const std::vector<int32_t> &sizes,
                      int32_t local_k)
{
    const int d = j->d;
    j->S = (int64_t)sizes.size();
    j->seg_off.assign(j->S + 1, 0);
    std::vector<int32_t> keff(j->S);
    for (int64_t s = 0; s < j->S; s++) {
        j->seg_off[s] = starts[s];
        keff[s] = std::min<int32_t>(local_k, sizes[s]);
    }
    j->seg_off[j->S] = j->n;
    TRY(build_lloyd_plan(j, j->lp, starts, sizes, keff));
    j->P = j->lp.P;
    job_free(j, j->cl);
    job_free(j, j->acc_l);
    job_free(j, j->cnt_l);
    j->cl = nullptr;
    j->acc_l = nullptr;
    j->cnt_l = nullptr;
    TRY(A(j, &j->cl, (size_t)j->P * d));
    TRY(A(j, &j->acc_l, (size_t)j->P * d));
    TRY(A(j, &j->cnt_l, 2 * (size_t)j->P));
    j->final_k = 0;              // the final plan depends on P
    return PSCL_OK;
}

static int plan_trace(pscl_job *j, int32_t iters)
{
    int64_t tl = j->trace ? (int64_t)iters * j->n : 0;
    if (tl != j->trace_l_len) {
        job_free(j, j->trace_l);
        j->trace_l = nullptr;
        j->trace_l_len = tl;
        if (tl) TRY(A(j, &j->trace_l, tl));
    }
    return PSCL_OK;
}

static int plan_cluster(pscl_job *j, int32_t final_k, int32_t iters, uint64_t seed, int prec)
{
    if (j->state < 2) return fail(PSCL_ESTATE, "pscl_cluster needs pscl_subcluster first");
    if (final_k < 1 || final_k > kMaxK) return fail(PSCL_EINVAL, "final_k=%d outside 1..%d", final_k, kMaxK);
    if ((int64_t)final_k > j->P)
        return fail(PSCL_EINVAL, "final_k=%d exceeds the %lld pooled local centers", final_k, (long long)j->P);
    if (iters < 0) return fail(PSCL_EINVAL, "iters < 0");
    TRY(check_prec(prec));
    const int d = j->d;
    j->fiters = iters;
    j->fseed = seed;
    j->fprec = prec;
    if (final_k != j->final_k) {
        drop_graph(j);
        j->final_k = final_k;
        std::vector<int64_t> starts(1, 0);
        std::vector<int32_t> sizes(1, (int32_t)j->P), keff(1, final_k);
        TRY(build_lloyd_plan(j, j->fp, starts, sizes, keff));
        job_free(j, j->cf);
        job_free(j, j->acc_f);
        job_free(j, j->cnt_f);
        job_free(j, j->lab_f);
        j->cf = nullptr;
        j->acc_f = nullptr;
        j->cnt_f = nullptr;
        j->lab_f = nullptr;
        // the SSE pass's tables for a search in chunks of 256 centers (tensor-core modes)
        {
            for (LloydPlan *q : {&j->sp256, &j->sprem, &j->fp256, &j->fprem}) {
                job_free(j, q->d_seg_start);
                job_free(j, q->d_i32);
                job_free(j, q->d_split);
                q->d_seg_start = nullptr;
                q->d_i32 = nullptr;
                q->d_split = nullptr;
            }
            std::vector<int64_t> s0(1, 0);
            std::vector<int32_t> sn(1, (int32_t)j->n);
            const int32_t rem = final_k % 256;
            if (final_k > 256) TRY(build_lloyd_plan(j, j->sp256, s0, sn, std::vector<int32_t>(1, 256)));
            if (final_k <= 256 || rem) TRY(build_lloyd_plan(j, j->sprem, s0, sn, std::vector<int32_t>(1, final_k <= 256 ? final_k : rem)));
            if (final_k > 256) {
                std::vector<int32_t> sp(1, (int32_t)j->P);
                TRY(build_lloyd_plan(j, j->fp256, s0, sp, std::vector<int32_t>(1, 256)));
                if (rem) TRY(build_lloyd_plan(j, j->fprem, s0, sp, std::vector<int32_t>(1, rem)));
            }
        }
        TRY(A(j, &j->cf, (size_t)final_k * d));
        TRY(A(j, &j->acc_f, (size_t)final_k * d));
        TRY(A(j, &j->cnt_f, 2 * (size_t)final_k));
        TRY(A(j, &j->lab_f, j->P));
    }
    if (!j->labels) {
        TRY(A(j, &j->labels, j->n));
        j->sse_blocks = sse_grid(j->n, j->ctx->sm_count);
        TRY(A(j, &j->blk_sse, j->sse_blocks));
        TRY(A(j, &j->sse, 1));
    }
    int64_t tl = j->trace ? (int64_t)iters * j->P : 0;
    if (tl != j->trace_f_len) {
        job_free(j, j->trace_f);
        j->trace_f = nullptr;
        j->trace_f_len = tl;
        if (tl) TRY(A(j, &j->trace_f, tl));
    }
    return PSCL_OK;
}

// ------------------------------------------------------------------ footprint
static size_t r256(size_t b) { return ((b ? b : 16) + 255) & ~(size_t)255; }

// Device bytes a job of this shape holds after pscl_run: every allocation of
// pscl_job_create, plan_subcluster and plan_cluster, each rounded as job_alloc rounds it.
static size_t job_footprint(int64_t n, int d, int64_t N, int local_k, int final_k, int iters, int dtype,
                            bool host_input, bool trace, int sm)
{
    size_t b = r256((size_t)n * d * 4) + 2 * r256((size_t)d * 8) + r256(scale_part_floats(n, d, sm) * 4) +
               r256(8 * 4) + r256(sizeof(PeelCtl)) + r256(kFlagWords * 4);
    if (dtype == PSCL_BF16) {
        b += r256((size_t)n * d * 4);                         // the widened points
        if (host_input) b += r256((size_t)n * d * 2);         // the bfloat16 copy
    } else if (host_input) {
        b += r256((size_t)n * d * 4);
    }
    const int64_t ord_ld = (n + 3) & ~(int64_t)3;
    const size_t nbk = peel_buckets(n);
    // rnd, pflag, ord, bcnt, bcs, lidx, kpos, band_k32, band_pos, gkey, gpos, akey, apos, pcnt,
    // perm, then xseg and the local labels
    b += r256((size_t)n * 4) + r256(2 * (size_t)n) + r256((size_t)d * ord_ld * 4) + r256((size_t)d * nbk * 4) +
         r256((size_t)d * nbk * 16) + 2 * r256(2 * (size_t)n * 4) + 2 * r256((size_t)n * 4) +
         r256((size_t)n * 8) + r256((size_t)n * 4) + r256((size_t)n * 8) + r256((size_t)n * 4) +
         r256(256 * (size_t)perm_grid(n, sm) * 4) + r256((size_t)n * 4) +
         r256((size_t)n * d * 4) + r256((size_t)n * 4);
    const int64_t S = (n + N - 1) / N;
    b += r256((size_t)S * d * 4);
    const int64_t tl = unit_target(n, sm, 0);
    int64_t units = 0, P = 0;
    for (int64_t s = 0; s < S; s++) {
        const int64_t m = std::min<int64_t>(N, n - s * N);
        units += (m + unit_size(m, tl) - 1) / unit_size(m, tl);
        P += std::min<int64_t>(local_k, m);
    }
    const size_t split = (size_t)10 * sm + 4;
    b += r256((size_t)S * 8) + r256((4 * (size_t)S + 3 * (size_t)units + 1) * 4) + r256(split * 4);
    b += r256((size_t)P * d * 4) + r256((size_t)P * d * 8) + r256(2 * (size_t)P * 4);
    if (trace) b += r256((size_t)iters * n * 4);
    const int64_t tf = unit_target(P, sm, 0);
    const int64_t uf = (P + unit_size(P, tf) - 1) / unit_size(P, tf);
    b += r256(8) + r256((4 + 3 * (size_t)uf + 1) * 4) + r256(split * 4);
    b += r256((size_t)final_k * d * 4) + r256((size_t)final_k * d * 8) + r256(2 * (size_t)final_k * 4) +
         r256((size_t)P * 4);
    {   // the SSE pass's row tables (one set of n rows; one or two of them)
        const int64_t tn = unit_target(n, sm, 0);
        const int64_t un = (n + unit_size(n, tn) - 1) / unit_size(n, tn);
        const int tables = (final_k > 256 ? 1 : 0) + (final_k <= 256 || final_k % 256 ? 1 : 0);
        b += (size_t)tables * (r256(8) + r256((4 + 3 * (size_t)un + 1) * 4) + r256(split * 4));
        if (final_k > 256) {   // the final Lloyd's, over the P pooled rows
            const int ftables = 1 + (final_k % 256 ? 1 : 0);
            const int64_t tp = unit_target(P, sm, 0);
            const int64_t up = (P + unit_size(P, tp) - 1) / unit_size(P, tp);
            b += (size_t)ftables * (r256(8) + r256((4 + 3 * (size_t)up + 1) * 4) + r256(split * 4));
        }
    }
    b += r256((size_t)n * 4) + r256((size_t)sse_grid(n, sm) * 8) + r256(8);
    if (trace) b += r256((size_t)iters * P * 4);
    return b;
}

cudaStream_t pscl::ctx_stream(const pscl_ctx *c) { return c->stream; }
int pscl::ctx_device(const pscl_ctx *c) { return c->device; }

int pscl::job_set_coop_stream(pscl_job *j, cudaStream_t s)
{
    for (int i = 0; i < 2; i++)
        if (!j->coop_ev[i]) CU(cudaEventCreateWithFlags(&j->coop_ev[i], cudaEventDisableTiming));
    j->coop = s;
    drop_graph(j);
    return PSCL_OK;
}

extern "C" int pscl_job_footprint(pscl_ctx *c, int64_t n, int32_t d, int64_t N, int32_t local_k, int32_t final_k,
                                  int32_t iters, int dtype, int points_on_device, int trace, size_t *bytes)
{
    if (!c || !bytes) return fail(PSCL_EINVAL, "ctx or bytes is NULL");
    if (n < 1 || d < 1 || N < 1 || local_k < 1 || final_k < 1 || iters < 0)
        return fail(PSCL_EINVAL, "shape out of range");
    if (dtype != PSCL_F32 && dtype != PSCL_BF16) return fail(PSCL_EINVAL, "unknown dtype %d", dtype);
    *bytes = job_footprint(n, d, N, local_k, final_k, iters, dtype, !points_on_device, trace != 0, c->sm_count);
    return PSCL_OK;
}

// Rows per thread of the float32 assignment: the option when set, else one row per thread
// when no unit has more rows than the kernel's 256 threads (small sets, e.g. the pooled
// local centers: more rows per thread would only score empty slots), else the default.
static int rows_per_thread(int option, const LloydPlan &p)
{
    return option ? option : (p.max_unit <= 256 ? 1 : 0);
}

// ------------------------------------------------------------------ enqueue (launches only)
static int run_lloyd(pscl_job *j, const LloydPlan &p, const float *pts, float *centers,
                     unsigned long long *acc, int32_t *cnt2, int32_t *labels, int32_t *trace,
                     int iters, uint64_t seed, uint32_t stage, bool plain, int prec,
                     const int32_t *weights = nullptr)
{
    cudaStream_t st = j->ctx->stream;
    const SegTable t = p.table();
    LloydBuffers b{};
    b.pts = pts;
    b.centers = centers;
    b.acc = acc;
    b.count = cnt2;
    b.labels = labels;
    b.trace = trace;
    b.rows = p.rows;
    b.weights = weights;
    // the near ties' candidate masks borrow the peel's bucket lists (d * ord_ld words, idle
    // once the peel is done; 8 words per row fit whenever d >= 8)
    if (j->pb.ord && (size_t)p.rows * 8 <= (size_t)j->d * (size_t)j->pb.ord_ld) b.tmask = j->pb.ord;
    // the pooled set past 256 centers: the chunked search's tables, its row state in the same
    // idle lists (4 rows + 1 words)
    if (stage == 1 && j->final_k > 256 && j->fp256.d_split && b.tmask &&
        (size_t)4 * p.rows + 1 <= (size_t)j->d * (size_t)j->pb.ord_ld) {
        b.chunk256 = j->fp256.table();
        b.chunkrem = (j->final_k % 256 ? j->fprem : j->fp256).table();
        b.has_chunks = true;
        b.chunk_scratch = j->pb.ord;
    }
    b.wait_limit = j->wait_limit;
    b.tc_stall = j->test_stall == 2;
    CU(launch_lloyd_init(b, t, j->d, p.P, seed, stage, j->first_k, p.kmax, st, &j->kt));
    if (!plain) {
        for (int it = 0; it < iters; it++) {
            b.count = cnt2 + (size_t)(it & 1) * p.P;
            CU(launch_lloyd_iter(b, cnt2 + (size_t)((it + 1) & 1) * p.P, t, j->d, it, 0, p.n_units, 0, p.P,
                                 p.kmax, prec, j->flags, j->ctx->sm_count, st, &j->kt, rows_per_thread(j->rpt, p)));
        }
    } else {
        for (int s = 0; s < p.n_seg; s++) {
            for (int it = 0; it < iters; it++) {
                b.count = cnt2 + (size_t)(it & 1) * p.P;
                CU(launch_lloyd_iter(b, cnt2 + (size_t)((it + 1) & 1) * p.P, t, j->d, it, p.seg_unit0[s],
                                     p.seg_unit0[s + 1], p.cen_off[s], (int64_t)p.cen_off[s] + p.k_eff[s],
                                     p.k_eff[s], prec, j->flags, j->ctx->sm_count, st, &j->kt,
                                     rows_per_thread(j->rpt, p)));
            }
        }
    }
    return PSCL_OK;
}

static int enqueue_scale(pscl_job *j, bool events)
{
    cudaStream_t st = j->ctx->stream;
    if (events) CU(cudaEventRecord(j->ev[0], st));
    CU(cudaMemsetAsync(j->flags, 0, kFlagWords * sizeof(uint32_t), st));   // errors and counters of this run
    if (j->dtype == PSCL_BF16) CU(launch_widen_bf16(j->in16, j->raw, j->n * j->d, j->ctx->sm_count, st));
    CU(launch_scale(j->dev_in, j->x, j->n, j->d, j->part, j->tickets, j->mn, j->mx, j->flags,
                    j->ctx->sm_count, st, &j->kt, j->dtype == PSCL_BF16));
    if (events) CU(cudaEventRecord(j->ev[1], st));
    return PSCL_OK;
}

static int enqueue_subcluster(pscl_job *j, bool events)
{
    cudaStream_t st = j->ctx->stream;
    j->pb.rounds_per_pass = j->peel_rounds;
    j->pb.wait_limit = j->wait_limit;
    j->pb.stall_first_barrier = j->test_stall == 1;
    j->pb.max_grid = j->peel_grid;
    if (j->coop) {
        CU(cudaEventRecord(j->coop_ev[0], st));
        CU(cudaStreamWaitEvent(j->coop, j->coop_ev[0], 0));
        CU(launch_peel(j->pb, j->n, j->d, j->N, j->ctx->sm_count, j->coop, &j->kt));
        CU(cudaEventRecord(j->coop_ev[1], j->coop));
        CU(cudaStreamWaitEvent(st, j->coop_ev[1], 0));
    } else {
        CU(launch_peel(j->pb, j->n, j->d, j->N, j->ctx->sm_count, st, &j->kt));
    }
    if (events) CU(cudaEventRecord(j->ev[2], st));
    TRY(run_lloyd(j, j->lp, j->pb.xseg, j->cl, j->acc_l, j->cnt_l, j->lab_l, j->trace_l, j->iters, j->seed, 0u,
                  j->plain != 0, j->prec));
    if (events) CU(cudaEventRecord(j->ev[3], st));
    return PSCL_OK;
}

static int enqueue_cluster(pscl_job *j, bool events)
{
    cudaStream_t st = j->ctx->stream;
    // count-weighted pooling: each local center weighs its cluster's size, the counts of
    // the last local iteration (left in its parity of the local count buffer)
    const int32_t *w = j->pool_w && j->iters > 0 ? j->cnt_l + (size_t)((j->iters - 1) & 1) * j->lp.P : nullptr;
    TRY(run_lloyd(j, j->fp, j->cl, j->cf, j->acc_f, j->cnt_f, j->lab_f, j->trace_f, j->fiters, j->fseed, 1u,
                  false, j->fprec, w));
    if (events) CU(cudaEventRecord(j->ev[4], st));
    // the SSE pass: on the tensor cores in chunks of 256 centers where the mode and the shape
    // allow (its row state borrows the peel's bucket lists, idle by now), else float32
    if (j->fprec != PSCL_PREC_FP32 && j->pb.ord && tc_sse_supported(j->d, j->final_k, j->fprec) &&
        (size_t)4 * j->n + 1 <= (size_t)j->d * (size_t)j->pb.ord_ld && j->n < ((int64_t)1 << 31)) {
        const SegTable t256 = (j->final_k > 256 ? j->sp256 : j->sprem).table();
        const SegTable trem = (j->final_k <= 256 || j->final_k % 256 ? j->sprem : j->sp256).table();
        CU(launch_final_sse_tc(j->x, j->n, j->d, j->cf, j->final_k, t256, trem, j->pb.ord, j->labels, j->blk_sse,
                               j->sse, j->tickets + 1, j->fprec, j->flags, j->wait_limit, j->ctx->sm_count, st,
                               &j->kt));
    } else {
        CU(launch_final_sse(j->x, j->n, j->d, j->cf, j->final_k, j->labels, j->blk_sse, j->sse, j->tickets + 1,
                            j->ctx->sm_count, st, &j->kt));
    }
    if (events) CU(cudaEventRecord(j->ev[5], st));
    return PSCL_OK;
}

// Count launches of a new run; bracket them with events if timing is on and the run is
// not being recorded into a graph.
static int timer_start(pscl_job *j, bool recording)
{
    KTimer &k = j->kt;
    k.reset();
    if (j->ktiming && !recording) {
        if (!k.ev) {
            k.cap = 1 << 14;
            k.ev = new cudaEvent_t[2 * k.cap];
            k.tag = new int[k.cap];
            for (int i = 0; i < 2 * k.cap; i++) CU(cudaEventCreate(&k.ev[i]));
        }
        k.n = 0;
    } else if (k.ev) {
        k.n = k.cap;                 // keep the events but record none
    }
    return PSCL_OK;
}

// ------------------------------------------------------------------ method entry points
extern "C" int pscl_scale_features(pscl_job *j)
{
    if (!j) return fail(PSCL_EINVAL, "job is NULL");
    CU(cudaSetDevice(j->ctx->device));
    TRY(timer_start(j, false));
    TRY(enqueue_scale(j, true));
    j->state = 1;
    j->ev_ok = false;
    return PSCL_OK;
}

extern "C" int pscl_subcluster(pscl_job *j, int64_t N, int32_t local_k, int32_t iters, uint64_t seed, int prec)
{
    if (!j) return fail(PSCL_EINVAL, "job is NULL");
    if (j->state < 1) return fail(PSCL_ESTATE, "pscl_subcluster needs pscl_scale_features first");
    CU(cudaSetDevice(j->ctx->device));
    TRY(plan_subcluster(j, N, local_k, iters, seed, prec));
    TRY(enqueue_subcluster(j, true));
    j->state = 2;
    return PSCL_OK;
}

extern "C" int pscl_subcluster_unequal(pscl_job *j, int32_t m, int32_t local_k, int32_t iters, uint64_t seed,
                                       int prec)
{
    if (!j) return fail(PSCL_EINVAL, "job is NULL");
    if (j->state < 1) return fail(PSCL_ESTATE, "pscl_subcluster_unequal needs pscl_scale_features first");
    if (m < 1 || m > kMaxLandmarks) return fail(PSCL_EINVAL, "m=%d outside 1..%d", m, kMaxLandmarks);
    if (local_k < 1 || local_k > kMaxK) return fail(PSCL_EINVAL, "local_k=%d outside 1..%d", local_k, kMaxK);
    if (iters < 0) return fail(PSCL_EINVAL, "iters < 0");
    TRY(check_prec(prec));
    CU(cudaSetDevice(j->ctx->device));
    TRY(alloc_subcluster_buffers(j));
    const int64_t n = j->n;
    const int d = j->d;
    cudaStream_t st = j->ctx->stream;
    drop_graph(j);
    if (m != j->unequal_m) {
        for (void *p : {(void *)j->u_lm, (void *)j->u_group, (void *)j->u_cnt, (void *)j->u_total, (void *)j->u_lo,
                        (void *)j->u_hi})
            job_free(j, p);
        j->u_lm = nullptr;
        j->u_group = nullptr;
        j->u_cnt = nullptr;
        j->u_total = nullptr;
        j->u_lo = j->u_hi = nullptr;
        TRY(A(j, &j->u_lm, (size_t)m * d));
        TRY(A(j, &j->u_group, n));
        TRY(A(j, &j->u_cnt, group_cnt_words(n, m)));
        TRY(A(j, &j->u_total, m));
        TRY(A(j, &j->u_lo, d));
        TRY(A(j, &j->u_hi, d));
        j->unequal_m = m;
    }
    // L, H of the scaled points, the landmarks, the groups and the grouped order
    CU(launch_minmax(j->x, n, d, j->part, j->tickets + 2, j->u_lo, j->u_hi, j->flags, j->ctx->sm_count, st, &j->kt));
    CU(launch_group_unequal(j->x, n, d, j->u_lo, j->u_hi, m, j->u_lm, j->u_group, j->u_cnt, j->u_total, j->pb.perm,
                            st, &j->kt));
    CU(launch_gather(j->x, j->pb.perm, n, d, j->pb.xseg, j->ctx->sm_count, st, &j->kt));
    // the subclusters are the groups that got points: their sizes decide the Lloyd plan
    std::vector<uint32_t> total(m);
    CU(cudaMemcpyAsync(total.data(), j->u_total, m * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    std::vector<int64_t> starts;
    std::vector<int32_t> sizes;
    int64_t off = 0;
    for (int i = 0; i < m; i++) {
        if (!total[i]) continue;
        starts.push_back(off);
        sizes.push_back((int32_t)total[i]);
        off += total[i];
    }
    if (off != n) return fail(PSCL_ECUDA, "internal error: the groups hold %lld of %lld points", (long long)off,
                              (long long)n);
    j->N = -(int64_t)m;                 // no equal-sized plan is current
    j->local_k = local_k;
    j->iters = iters;
    j->seed = seed;
    j->prec = prec;
    TRY(plan_local(j, starts, sizes, local_k));
    TRY(plan_trace(j, iters));
    TRY(run_lloyd(j, j->lp, j->pb.xseg, j->cl, j->acc_l, j->cnt_l, j->lab_l, j->trace_l, iters, seed, 0u,
                  j->plain != 0, prec));
    j->state = 2;
    j->ev_ok = false;
    return PSCL_OK;
}

extern "C" int pscl_cluster(pscl_job *j, int32_t final_k, int32_t iters, uint64_t seed, int prec)
{
    if (!j) return fail(PSCL_EINVAL, "job is NULL");
    CU(cudaSetDevice(j->ctx->device));
    TRY(plan_cluster(j, final_k, iters, seed, prec));
    TRY(enqueue_cluster(j, true));
    j->state = 3;
    j->ev_ok = true;
    return PSCL_OK;
}

extern "C" int pscl_run(pscl_job *j, int64_t N, int32_t local_k, int32_t final_k, int32_t iters,
                        uint64_t seed, int prec)
{
    if (!j) return fail(PSCL_EINVAL, "job is NULL");
    CU(cudaSetDevice(j->ctx->device));
    // planning (allocation, table uploads) happens outside any recording
    j->state = 1;
    TRY(plan_subcluster(j, N, local_k, iters, seed, prec));
    j->state = 2;
    TRY(plan_cluster(j, final_k, iters, seed, prec));
    cudaStream_t st = j->ctx->stream;
    if (!j->graph) {
        TRY(timer_start(j, false));
        TRY(enqueue_scale(j, true));
        TRY(enqueue_subcluster(j, true));
        TRY(enqueue_cluster(j, true));
        j->state = 3;
        j->ev_ok = true;
        return PSCL_OK;
    }
    uint64_t key[8] = {(uint64_t)N, (uint64_t)local_k, (uint64_t)final_k, (uint64_t)iters, seed, (uint64_t)prec,
                       (uint64_t)(uintptr_t)j->dev_in ^ (uint64_t)(uintptr_t)j->in16,
                       (uint64_t)(j->plain | j->trace << 1 | j->first_k << 2 | j->rpt << 3 | j->pool_w << 5)};
    if (j->gexec && memcmp(key, j->gkey, sizeof key) != 0) drop_graph(j);
    if (!j->gexec) {
        cudaGraph_t g = nullptr;
        TRY(timer_start(j, true));
        CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_scale(j, false);
        if (!rc) rc = enqueue_subcluster(j, false);
        if (!rc) rc = enqueue_cluster(j, false);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(PSCL_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&j->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            j->gexec = nullptr;
            return fail(PSCL_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
        }
        memcpy(j->gkey, key, sizeof key);
    }
    CU(cudaGraphLaunch(j->gexec, st));
    j->state = 3;
    j->ev_ok = false;
    return PSCL_OK;
}

extern "C" int pscl_job_sync(pscl_job *j)
{
    if (!j) return fail(PSCL_EINVAL, "job is NULL");
    CU(cudaSetDevice(j->ctx->device));
    CU(cudaStreamSynchronize(j->ctx->stream));
    uint32_t h[kFlagWords];
    CU(cudaMemcpy(h, j->flags, sizeof h, cudaMemcpyDeviceToHost));
    if (h[0]) return fail(PSCL_EINVAL, "the input holds a value that is not finite");
    if (h[1] & 2u) return fail(PSCL_ETIMEOUT, "a bounded device-side wait gave up (peel barrier)");
    if (h[1] & 4u) return fail(PSCL_ETIMEOUT, "a bounded device-side wait gave up (tensor-core commit)");
    if (h[1] & 1u) return fail(PSCL_ECUDA, "internal error: the peel's float32 filter bound was contradicted");
    return PSCL_OK;
}

// ------------------------------------------------------------------ results
extern "C" int pscl_get_scaled(pscl_job *j, float *out)
{
    TRY(pscl_job_sync(j));
    if (j->state < 1) return fail(PSCL_ESTATE, "not scaled");
    if (out) CU(cudaMemcpy(out, j->x, (size_t)j->n * j->d * sizeof(float), cudaMemcpyDeviceToHost));
    return PSCL_OK;
}

extern "C" int pscl_get_sizes(pscl_job *j, int64_t *n_seg, int64_t *n_pooled)
{
    if (!j) return fail(PSCL_EINVAL, "job is NULL");
    if (j->state < 2) return fail(PSCL_ESTATE, "no subcluster plan yet");
    if (n_seg) *n_seg = j->S;
    if (n_pooled) *n_pooled = j->P;
    return PSCL_OK;
}

extern "C" int pscl_get_partition(pscl_job *j, int64_t *perm, int64_t *seg_off, int64_t *n_seg)
{
    TRY(pscl_job_sync(j));
    if (j->state < 2) return fail(PSCL_ESTATE, "not subclustered");
    if (perm) {
        std::vector<uint32_t> h(j->n);
        CU(cudaMemcpy(h.data(), j->pb.perm, j->n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < j->n; i++) perm[i] = h[i];
    }
    if (seg_off) memcpy(seg_off, j->seg_off.data(), (j->S + 1) * sizeof(int64_t));
    if (n_seg) *n_seg = j->S;
    return PSCL_OK;
}

extern "C" int pscl_get_local_centers(pscl_job *j, float *centers, int32_t *k_eff, int32_t *counts)
{
    TRY(pscl_job_sync(j));
    if (j->state < 2) return fail(PSCL_ESTATE, "not subclustered");
    if (centers) CU(cudaMemcpy(centers, j->cl, (size_t)j->P * j->d * sizeof(float), cudaMemcpyDeviceToHost));
    if (k_eff) memcpy(k_eff, j->lp.k_eff.data(), j->S * sizeof(int32_t));
    if (counts) {
        if (j->iters == 0) {
            memset(counts, 0, j->P * sizeof(int32_t));
        } else {
            const int32_t *src = j->cnt_l + (size_t)((j->iters - 1) & 1) * j->P;
            CU(cudaMemcpy(counts, src, j->P * sizeof(int32_t), cudaMemcpyDeviceToHost));
        }
    }
    return PSCL_OK;
}

extern "C" int pscl_get_result(pscl_job *j, float *centers, int32_t *labels, double *sse)
{
    TRY(pscl_job_sync(j));
    if (j->state < 3) return fail(PSCL_ESTATE, "not clustered");
    if (centers) CU(cudaMemcpy(centers, j->cf, (size_t)j->final_k * j->d * sizeof(float), cudaMemcpyDeviceToHost));
    if (labels) CU(cudaMemcpy(labels, j->labels, j->n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (sse) CU(cudaMemcpy(sse, j->sse, sizeof(double), cudaMemcpyDeviceToHost));
    return PSCL_OK;
}

extern "C" int pscl_get_label_trace(pscl_job *j, int stage, int32_t *out)
{
    TRY(pscl_job_sync(j));
    if (!out) return fail(PSCL_EINVAL, "out is NULL");
    if (stage == 0) {
        if (j->state < 2 || !j->trace_l) return fail(PSCL_ESTATE, "no local label trace recorded");
        CU(cudaMemcpy(out, j->trace_l, j->trace_l_len * sizeof(int32_t), cudaMemcpyDeviceToHost));
    } else if (stage == 1) {
        if (j->state < 3 || !j->trace_f) return fail(PSCL_ESTATE, "no final label trace recorded");
        CU(cudaMemcpy(out, j->trace_f, j->trace_f_len * sizeof(int32_t), cudaMemcpyDeviceToHost));
    } else {
        return fail(PSCL_EINVAL, "stage must be 0 or 1");
    }
    return PSCL_OK;
}

extern "C" int pscl_get_kernel_times(pscl_job *j, int64_t *launches, float *ms)
{
    TRY(pscl_job_sync(j));
    if (launches)
        for (int i = 0; i < PSCL_K_COUNT; i++) launches[i] = j->kt.launches[i];
    if (ms) {
        for (int i = 0; i < PSCL_K_COUNT; i++) ms[i] = 0.0f;
        const int used = j->kt.ev && j->ktiming ? std::min(j->kt.n, j->kt.cap) : 0;
        for (int e = 0; e < used; e++) {
            float t = 0.0f;
            CU(cudaEventElapsedTime(&t, j->kt.ev[2 * e], j->kt.ev[2 * e + 1]));
            ms[j->kt.tag[e]] += t;
        }
    }
    return PSCL_OK;
}

extern "C" int pscl_get_recheck_stats(pscl_job *j, int64_t *rechecked, int64_t *assigned)
{
    TRY(pscl_job_sync(j));
    uint32_t h[kFlagWords];
    CU(cudaMemcpy(h, j->flags, sizeof h, cudaMemcpyDeviceToHost));
    if (rechecked) *rechecked = h[2];
    if (assigned) *assigned = h[3];
    return PSCL_OK;
}

extern "C" int pscl_get_peel_stats(pscl_job *j, int64_t *epochs, int64_t *passes, int64_t *key_updates,
                                   int64_t *barriers)
{
    TRY(pscl_job_sync(j));
    if (!j->pb.ctl) return fail(PSCL_ESTATE, "no equal-sized subclustering has run on this job");
    uint32_t v[4];
    static_assert(offsetof(PeelCtl, passes) == offsetof(PeelCtl, epochs) + 4 &&
                      offsetof(PeelCtl, key_updates) == offsetof(PeelCtl, epochs) + 8 &&
                      offsetof(PeelCtl, barriers) == offsetof(PeelCtl, epochs) + 12,
                  "the statistics are adjacent");
    CU(cudaMemcpy(v, reinterpret_cast<const char *>(j->pb.ctl) + offsetof(PeelCtl, epochs), sizeof v,
                  cudaMemcpyDeviceToHost));
    if (epochs) *epochs = v[0];
    if (passes) *passes = v[1];
    if (key_updates) *key_updates = v[2];
    if (barriers) *barriers = v[3];
    return PSCL_OK;
}

extern "C" int pscl_measure_grid_barrier(int device, double *us)
{
    if (!us) return fail(PSCL_EINVAL, "us is NULL");
    CU(cudaSetDevice(device));
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    bool timed_out = false;
    CU(measure_grid_barrier(sms, us, &timed_out));
    if (timed_out) return fail(PSCL_ETIMEOUT, "a barrier of the measurement gave up");
    return PSCL_OK;
}

extern "C" int pscl_get_phase_ms(pscl_job *j, float *ms)
{
    TRY(pscl_job_sync(j));
    if (!ms) return fail(PSCL_EINVAL, "ms is NULL");
    if (!j->ev_ok) return fail(PSCL_ESTATE, "no timed run (phase times need an unrecorded pscl_run or the three calls)");
    for (int i = 0; i < 5; i++) CU(cudaEventElapsedTime(&ms[i], j->ev[i], j->ev[i + 1]));
    return PSCL_OK;
}

// ------------------------------------------------------------------ uneven batch
// Independent point sets, each min-max scaled on its own and clustered by its own seeded
// Lloyd run; every launch covers all sets (work units of at most 1024 rows of one set),
// and a run is recorded once into a CUDA graph.
struct pscl_batch : Owner {
    int d = 0, n_inst = 0;
    int64_t rows = 0;
    std::vector<int64_t> starts;
    std::vector<int32_t> sizes, keff;
    const float *dev_in = nullptr;
    float *raw = nullptr, *x = nullptr, *part = nullptr;
    double *mn = nullptr, *mx = nullptr;
    LloydPlan plan;
    float *centers = nullptr;
    unsigned long long *acc = nullptr;
    int32_t *cnt = nullptr, *labels = nullptr, *out_labels = nullptr, *trace = nullptr;
    uint32_t *tmask = nullptr;        // rows x 8 (tensor-core precisions only)
    int64_t trace_len = 0;
    double *unit_sse = nullptr, *seg_sse = nullptr;
    uint32_t *flags = nullptr;
    int64_t unit_rows = 0;            // 0: the planner's default
    int rpt = 0;                      // rows per thread of the float32 kernel, 0 = default
    int trace_on = 0, graph = 1, plain = 0;
    int iters = 0;
    KTimer kt;
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey[6] = {};
    cudaEvent_t ev[2] = {};
};

static void batch_drop_graph(pscl_batch *b)
{
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
}

// (Re)build the work-unit plan and everything sized by it.
static int batch_plan(pscl_batch *b)
{
    batch_drop_graph(b);
    TRY(build_lloyd_plan(b, b->plan, b->starts, b->sizes, b->keff, b->unit_rows));
    job_free(b, b->part);
    job_free(b, b->unit_sse);
    b->part = nullptr;
    b->unit_sse = nullptr;
    TRY(A(b, &b->part, 2 * (size_t)b->plan.n_units * b->d));
    TRY(A(b, &b->unit_sse, b->plan.n_units));
    return PSCL_OK;
}

extern "C" int pscl_batch_create(pscl_ctx *c, const void *points, int on_device, int32_t d, int32_t n_inst,
                                 const int64_t *sizes, const int32_t *k, pscl_batch **out)
{
    if (!c || !out || !points || !sizes || !k) return fail(PSCL_EINVAL, "a required pointer is NULL");
    if (d < 1 || d > kMaxD) return fail(PSCL_EINVAL, "d=%d outside 1..%d", d, kMaxD);
    if (n_inst < 1) return fail(PSCL_EINVAL, "n_inst=%d < 1", n_inst);
    int64_t rows = 0;
    for (int i = 0; i < n_inst; i++) {
        if (sizes[i] < 1 || sizes[i] > (int64_t)INT32_MAX)
            return fail(PSCL_EINVAL, "instance %d: size %lld outside 1..2^31-1", i, (long long)sizes[i]);
        if (k[i] < 1 || k[i] > kMaxK) return fail(PSCL_EINVAL, "instance %d: k=%d outside 1..%d", i, k[i], kMaxK);
        rows += sizes[i];
    }
    if (rows > (int64_t)INT32_MAX) return fail(PSCL_EINVAL, "%lld rows in all exceed 2^31-1", (long long)rows);
    CU(cudaSetDevice(c->device));
    pscl_batch *b = new pscl_batch();
    b->ctx = c;
    b->d = d;
    b->n_inst = n_inst;
    b->rows = rows;
    b->starts.resize(n_inst);
    b->sizes.resize(n_inst);
    b->keff.resize(n_inst);
    int64_t P = 0, off = 0;
    for (int i = 0; i < n_inst; i++) {
        b->starts[i] = off;
        b->sizes[i] = (int32_t)sizes[i];
        b->keff[i] = (int32_t)std::min<int64_t>(k[i], sizes[i]);
        off += sizes[i];
        P += b->keff[i];
    }
    int rc = PSCL_OK;
    if (on_device) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, points) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
            at.device != c->device || ((uintptr_t)points & 15) != 0) {
            cudaGetLastError();
            rc = fail(PSCL_EINVAL, "points_on_device=1 but the pointer is not 16-byte aligned device memory of device %d",
                      c->device);
        }
        b->dev_in = static_cast<const float *>(points);
    } else {
        rc = A(b, &b->raw, (size_t)rows * d);
        if (!rc && cudaMemcpyAsync(b->raw, points, (size_t)rows * d * sizeof(float), cudaMemcpyHostToDevice,
                                   c->stream) != cudaSuccess)
            rc = fail(PSCL_ECUDA, "upload of the points failed");
        b->dev_in = b->raw;
    }
    if (!rc) rc = A(b, &b->x, (size_t)rows * d);
    if (!rc) rc = A(b, &b->mn, (size_t)n_inst * d);
    if (!rc) rc = A(b, &b->mx, (size_t)n_inst * d);
    if (!rc) rc = A(b, &b->centers, (size_t)P * d);
    if (!rc) rc = A(b, &b->acc, (size_t)P * d);
    if (!rc) rc = A(b, &b->cnt, 2 * (size_t)P);
    if (!rc) rc = A(b, &b->labels, rows);
    if (!rc) rc = A(b, &b->out_labels, rows);
    if (!rc) rc = A(b, &b->seg_sse, n_inst);
    if (!rc) rc = A(b, &b->flags, kFlagWords);
    if (!rc) rc = batch_plan(b);
    for (int i = 0; i < 2 && !rc; i++)
        if (cudaEventCreate(&b->ev[i]) != cudaSuccess) rc = fail(PSCL_ECUDA, "cudaEventCreate failed");
    if (rc) {
        std::string msg = g_err;
        pscl_batch_destroy(b);
        g_err = msg;
        return rc;
    }
    *out = b;
    return PSCL_OK;
}

extern "C" int pscl_batch_load(pscl_batch *b, const void *points, int on_device)
{
    if (!b || !points) return fail(PSCL_EINVAL, "batch or points is NULL");
    CU(cudaSetDevice(b->ctx->device));
    if (on_device) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, points) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
            at.device != b->ctx->device || ((uintptr_t)points & 15) != 0) {
            cudaGetLastError();
            return fail(PSCL_EINVAL, "points_on_device=1 but the pointer is not 16-byte aligned device memory of device %d",
                        b->ctx->device);
        }
        if (b->dev_in != points) batch_drop_graph(b);
        b->dev_in = static_cast<const float *>(points);
        return PSCL_OK;
    }
    if (!b->raw) TRY(A(b, &b->raw, (size_t)b->rows * b->d));
    if (b->dev_in != b->raw) batch_drop_graph(b);
    CU(cudaMemcpyAsync(b->raw, points, (size_t)b->rows * b->d * sizeof(float), cudaMemcpyHostToDevice, b->ctx->stream));
    b->dev_in = b->raw;
    return PSCL_OK;
}

extern "C" int pscl_batch_destroy(pscl_batch *b)
{
    if (!b) return fail(PSCL_EINVAL, "batch is NULL");
    cudaSetDevice(b->ctx->device);
    cudaStreamSynchronize(b->ctx->stream);
    batch_drop_graph(b);
    for (auto &a : b->allocs) {
        cudaFreeAsync(a.p, b->ctx->stream);
        b->ctx->in_use -= a.bytes;
    }
    for (int i = 0; i < 2; i++)
        if (b->ev[i]) cudaEventDestroy(b->ev[i]);
    delete b;
    return PSCL_OK;
}

extern "C" int pscl_batch_set_option(pscl_batch *b, int opt, int64_t v)
{
    if (!b) return fail(PSCL_EINVAL, "batch is NULL");
    switch (opt) {
    case PSCL_OPT_TRACE_LABELS: b->trace_on = v != 0; break;
    case PSCL_OPT_GRAPH: b->graph = v != 0; break;
    case PSCL_OPT_PLAIN_LLOYD: b->plain = v != 0; break;
    case PSCL_OPT_UNIT_ROWS:
        if (v < 0 || v > 1024) return fail(PSCL_EINVAL, "unit rows %lld outside 0..1024", (long long)v);
        b->unit_rows = v;
        return batch_plan(b);
    case PSCL_OPT_ROWS_PER_THREAD:
        if (v < 0 || v > 2) return fail(PSCL_EINVAL, "rows per thread must be 0, 1 or 2");
        b->rpt = (int)v;
        break;
    default: return fail(PSCL_EINVAL, "option %d does not apply to a batch", opt);
    }
    batch_drop_graph(b);
    return PSCL_OK;
}

// Scale, seeded init (stage 0, segment = instance), `iters` iterations, per-instance SSE.
static int batch_enqueue(pscl_batch *b, int iters, uint64_t seed, int prec, bool events)
{
    cudaStream_t st = b->ctx->stream;
    b->kt.reset();                     // a recorded run keeps the count of its recording
    const SegTable t = b->plan.table();
    const int32_t *u0 = b->plan.d_unit0();
    CU(cudaMemsetAsync(b->flags, 0, kFlagWords * sizeof(uint32_t), st));
    CU(launch_seg_scale(b->dev_in, b->x, t, u0, b->d, b->part, b->mn, b->mx, b->flags, st, &b->kt));
    LloydBuffers lb{};
    lb.pts = b->x;
    lb.centers = b->centers;
    lb.acc = b->acc;
    lb.count = b->cnt;
    lb.labels = b->labels;
    lb.trace = b->trace_on ? b->trace : nullptr;
    lb.rows = b->rows;
    lb.tmask = b->tmask;
    const int64_t P = b->plan.P;
    CU(launch_lloyd_init(lb, t, b->d, P, seed, 0u, 0, b->plan.kmax, st, &b->kt));
    if (events) CU(cudaEventRecord(b->ev[0], st));
    if (!b->plain) {
        for (int it = 0; it < iters; it++) {
            lb.count = b->cnt + (size_t)(it & 1) * P;
            CU(launch_lloyd_iter(lb, b->cnt + (size_t)((it + 1) & 1) * P, t, b->d, it, 0, b->plan.n_units, 0, P,
                                 b->plan.kmax, prec, b->flags, b->ctx->sm_count, st, &b->kt,
                                 rows_per_thread(b->rpt, b->plan)));
        }
    } else {                           // one launch pair per instance and iteration
        const LloydPlan &p = b->plan;
        for (int s = 0; s < p.n_seg; s++) {
            for (int it = 0; it < iters; it++) {
                lb.count = b->cnt + (size_t)(it & 1) * P;
                CU(launch_lloyd_iter(lb, b->cnt + (size_t)((it + 1) & 1) * P, t, b->d, it, p.seg_unit0[s],
                                     p.seg_unit0[s + 1], p.cen_off[s], (int64_t)p.cen_off[s] + p.k_eff[s], p.k_eff[s],
                                     prec, b->flags, b->ctx->sm_count, st, &b->kt, rows_per_thread(b->rpt, p)));
            }
        }
    }
    if (events) CU(cudaEventRecord(b->ev[1], st));
    CU(launch_seg_sse(b->x, t, u0, b->d, b->centers, b->plan.kmax, b->out_labels, b->unit_sse, b->seg_sse, st,
                      &b->kt));
    return PSCL_OK;
}

extern "C" int pscl_batch_run(pscl_batch *b, int32_t iters, uint64_t seed, int prec)
{
    if (!b) return fail(PSCL_EINVAL, "batch is NULL");
    if (iters < 0) return fail(PSCL_EINVAL, "iters < 0");
    TRY(check_prec(prec));
    CU(cudaSetDevice(b->ctx->device));
    int64_t tl = b->trace_on ? (int64_t)iters * b->rows : 0;
    if (tl != b->trace_len) {
        batch_drop_graph(b);
        job_free(b, b->trace);
        b->trace = nullptr;
        b->trace_len = tl;
        if (tl) TRY(A(b, &b->trace, tl));
    }
    b->iters = iters;
    // the tensor-core assignment's candidate masks: 8 words per row, allocated once
    if (prec != PSCL_PREC_FP32 && !b->tmask) TRY(A(b, &b->tmask, (size_t)b->rows * 8));
    if (!b->graph) return batch_enqueue(b, iters, seed, prec, true);
    const uint64_t key[6] = {(uint64_t)iters, seed, (uint64_t)prec, (uint64_t)(b->trace_on | b->plain << 1),
                             (uint64_t)b->unit_rows, (uint64_t)b->rpt};
    if (b->gexec && memcmp(key, b->gkey, sizeof key) != 0) batch_drop_graph(b);
    cudaStream_t st = b->ctx->stream;
    if (!b->gexec) {
        cudaGraph_t g = nullptr;
        CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = batch_enqueue(b, iters, seed, prec, false);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(PSCL_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->gexec = nullptr;
            return fail(PSCL_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
        }
        memcpy(b->gkey, key, sizeof key);
    }
    CU(cudaGraphLaunch(b->gexec, st));
    return PSCL_OK;
}

extern "C" int pscl_batch_sync(pscl_batch *b)
{
    if (!b) return fail(PSCL_EINVAL, "batch is NULL");
    CU(cudaSetDevice(b->ctx->device));
    CU(cudaStreamSynchronize(b->ctx->stream));
    uint32_t h[kFlagWords];
    CU(cudaMemcpy(h, b->flags, sizeof h, cudaMemcpyDeviceToHost));
    if (h[0]) return fail(PSCL_EINVAL, "the input holds a value that is not finite");
    if (h[1] & 4u) return fail(PSCL_ETIMEOUT, "a bounded device-side wait gave up (tensor-core commit)");
    return PSCL_OK;
}

extern "C" int pscl_batch_get(pscl_batch *b, float *centers, int32_t *labels, double *sse)
{
    TRY(pscl_batch_sync(b));
    if (centers) CU(cudaMemcpy(centers, b->centers, (size_t)b->plan.P * b->d * sizeof(float), cudaMemcpyDeviceToHost));
    if (labels) CU(cudaMemcpy(labels, b->out_labels, (size_t)b->rows * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (sse) CU(cudaMemcpy(sse, b->seg_sse, (size_t)b->n_inst * sizeof(double), cudaMemcpyDeviceToHost));
    return PSCL_OK;
}

extern "C" int pscl_batch_get_scaled(pscl_batch *b, float *out)
{
    TRY(pscl_batch_sync(b));
    if (!out) return fail(PSCL_EINVAL, "out is NULL");
    CU(cudaMemcpy(out, b->x, (size_t)b->rows * b->d * sizeof(float), cudaMemcpyDeviceToHost));
    return PSCL_OK;
}

extern "C" int pscl_batch_get_label_trace(pscl_batch *b, int32_t *out)
{
    TRY(pscl_batch_sync(b));
    if (!out) return fail(PSCL_EINVAL, "out is NULL");
    if (!b->trace_len) return fail(PSCL_ESTATE, "no label trace was recorded (PSCL_OPT_TRACE_LABELS)");
    CU(cudaMemcpy(out, b->trace, (size_t)b->trace_len * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return PSCL_OK;
}

extern "C" int pscl_batch_launches(pscl_batch *b, int64_t *launches)
{
    if (!b || !launches) return fail(PSCL_EINVAL, "batch or launches is NULL");
    int64_t t = 0;
    for (int i = 0; i < PSCL_K_COUNT; i++) t += b->kt.launches[i];
    *launches = t;
    return PSCL_OK;
}

extern "C" int pscl_batch_lloyd_ms(pscl_batch *b, float *ms)
{
    TRY(pscl_batch_sync(b));
    if (!ms) return fail(PSCL_EINVAL, "ms is NULL");
    if (b->graph) return fail(PSCL_ESTATE, "Lloyd time is kept only for runs outside a graph (PSCL_OPT_GRAPH 0)");
    CU(cudaEventElapsedTime(ms, b->ev[0], b->ev[1]));
    return PSCL_OK;
}

// ------------------------------------------------------------------ autotuner
// Work-unit size and rows per thread of the assignment kernel, chosen by timing a few
// Lloyd iterations of the batch itself for every candidate.  Neither changes any result
// (the sums are exact integers), only the time.  Choices are remembered per (device, d,
// largest k, log2 of the rows, precision) for the life of the process.
struct TuneKey {
    int device, d, kmax, lg_rows, prec;
    bool operator==(const TuneKey &o) const
    {
        return device == o.device && d == o.d && kmax == o.kmax && lg_rows == o.lg_rows && prec == o.prec;
    }
};
struct TuneChoice {
    TuneKey key;
    int64_t unit_rows;
    int rpt;
};
static std::vector<TuneChoice> g_tuned;

extern "C" int pscl_batch_tune(pscl_batch *b, int32_t iters, int prec, int64_t *unit_rows, int32_t *rows_per_thread,
                               int32_t *cached)
{
    if (!b) return fail(PSCL_EINVAL, "batch is NULL");
    if (iters < 1) return fail(PSCL_EINVAL, "iters < 1");
    TRY(check_prec(prec));
    CU(cudaSetDevice(b->ctx->device));
    int lg = 0;
    while ((int64_t)1 << (lg + 1) <= b->rows) lg++;
    const TuneKey key{b->ctx->device, b->d, b->plan.kmax, lg, prec};
    int hit = 0;
    for (auto &c : g_tuned) {
        if (c.key == key) {
            b->unit_rows = c.unit_rows;
            b->rpt = c.rpt;
            hit = 1;
            break;
        }
    }
    if (!hit) {
        const int save_graph = b->graph, save_trace = b->trace_on;
        b->graph = 0;
        b->trace_on = 0;
        static const int64_t units[] = {128, 256, 512, 1024};
        float best = 0.0f;
        int64_t best_u = 0;
        int best_r = 0;
        for (int64_t u : units) {
            for (int r = 0; r < 3; r++) {
                b->unit_rows = u;
                b->rpt = r;
                TRY(batch_plan(b));
                TRY(pscl_batch_run(b, 1, 0, prec));           // warm-up
                TRY(pscl_batch_run(b, iters, 0, prec));
                float ms = 0.0f;
                TRY(pscl_batch_lloyd_ms(b, &ms));
                if (best_u == 0 || ms < best) {
                    best = ms;
                    best_u = u;
                    best_r = r;
                }
            }
        }
        b->graph = save_graph;
        b->trace_on = save_trace;
        b->unit_rows = best_u;
        b->rpt = best_r;
        g_tuned.push_back({key, best_u, best_r});
    }
    TRY(batch_plan(b));
    if (unit_rows) *unit_rows = b->unit_rows;
    if (rows_per_thread) *rows_per_thread = b->rpt;
    if (cached) *cached = hit;
    return PSCL_OK;
}
