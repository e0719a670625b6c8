// Internal declarations of the pscl CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pscl.h"

namespace pscl {

constexpr int kMaxD = 1024;          // attributes per point
constexpr int kMaxK = 4096;          // centers of one Lloyd run
constexpr int kHistBins = 2048;      // 11-bit radix digits of the peel's key select
constexpr int kFixShift = 32;        // fixed-point scale 2^32 of the centroid sums

constexpr int kMaxPeelGrid = 2048;   // CTAs of the persistent peel launch

// Rounds one peel epoch may select from one set of distances (boundaries per epoch).
constexpr int kMaxEpoch = 32;

// Device-resident control block of one persistent peel launch (cleared before it).
struct PeelCtl {
    uint32_t h0[kHistBins];              // first digit (key bits 31..21) of the live keys
    uint32_t h1[kMaxEpoch][kHistBins];   // second digit (bits 20..10) inside each boundary's bin
    uint32_t Lbits[kMaxD];               // landmark of the current epoch (float bits)
    uint32_t lptr[kMaxD];                // per attribute: buckets in front of it hold no remaining point
    uint32_t chold[kMaxD];               // live points whose attribute j equals L_j
    uint32_t hmax[kMaxD];                // the largest key among them (since the last pass)
    uint32_t hcnt[kMaxD][kMaxEpoch];     // of those, the ones assigned to each round of the epoch
    uint32_t cert[kMaxEpoch];            // points certainly in each round of the epoch
    uint32_t bnd[kMaxEpoch];             // band points settled into each round of the epoch
    uint32_t gcnt[kMaxEpoch];            // band entries of each group of boundaries
    uint32_t gfill[kMaxEpoch];           // of those, regrouped into the group's region so far
    uint32_t g_in[kMaxEpoch], g_out[kMaxEpoch];   // a group's band: keys in [g_in, g_out]
    uint32_t g_q1[kMaxEpoch], g_q2[kMaxEpoch];    // a group's first and last boundary
    float kref;                          // lower end of the first boundary's key bin, last epoch
    uint32_t n_slots;                    // first-digit bins with a second-digit histogram
    uint32_t n_groups;
    uint32_t band_cnt;                   // band entries listed this epoch
    uint32_t k_eff;                      // boundaries the epoch resolves (rounds it can commit)
    uint32_t k_commit;                   // rounds the epoch commits
    uint32_t l_changed;                  // the landmark changes after them
    uint32_t bar_count;                  // grid barrier: arrivals since the launch
    uint32_t abort;                      // set when a barrier wait gave up
    uint32_t epochs;                     // statistics: epochs run,
    uint32_t passes;                     //   distance passes over the points left,
    uint32_t key_updates;                //   of which updates of the keys in a few attributes,
    uint32_t barriers;                   //   grid-wide barriers passed
};

// v (a scaled coordinate, in [0, 1]) times 2^32 rounded to the nearest integer, ties to
// even, as hi 2^16 + lo with lo <= 2^16: s = v 2^16 is exact, hi = floor(s), the fraction
// s - hi and its product with 2^16 are exact, and only lo is rounded.  Two 32-bit
// conversions: the 64-bit float-to-integer conversion runs on the float64 pipe.
__device__ __forceinline__ void fix_parts(float v, uint32_t &hi, uint32_t &lo)
{
    const float s = v * 65536.0f;
    hi = __float2uint_rz(s);
    lo = __float2uint_rn((s - __uint2float_rz(hi)) * 65536.0f);
}

__device__ __forceinline__ unsigned long long fix_of(float v)
{
    uint32_t hi, lo;
    fix_parts(v, hi, lo);
    return ((unsigned long long)hi << 16) + lo;
}

// Job flags read by the host at every synchronisation.
//   [0] != 0: an input value is not finite
//   [1] bit 0: the peel's float32 bound was contradicted (internal error)
//       bit 1: a bounded device-side wait gave up (peel barrier)
//       bit 2: a bounded device-side wait gave up (tensor-core commit)
//   [2] rows the tensor-core assignment re-scored in float32 (near ties)
//   [3] rows the tensor-core assignment assigned
constexpr int kFlagWords = 4;

// Segment table of one batched Lloyd launch (device arrays).
struct SegTable {
    const int64_t *seg_start;        // first row of each segment in the packed points
    const int32_t *seg_size;
    const int32_t *cen_off;          // first center of each segment
    const int32_t *k_eff;            // centers of each segment
    const int32_t *unit_seg;         // work units: segment, first row (relative), rows
    const int32_t *unit_start;
    const int32_t *unit_count;
    int n_seg;
    int n_units;
    // Persistent launches over all units with m CTAs per SM (m = 1..4): CTA c serves the
    // units [split[split_off[m] + c], split[split_off[m] + c + 1]) (NULL: no split).
    const int32_t *split;
    int split_off[5];
};

// Launch bookkeeping: every launcher counts its launches per pscl_kernel tag and, when
// `ev` is set, brackets each launch with a pair of CUDA events on the stream.
struct KTimer {
    int64_t launches[PSCL_K_COUNT] = {};
    cudaEvent_t *ev = nullptr;       // 2 * cap events, or NULL (count only)
    int *tag = nullptr;
    int cap = 0;
    int n = 0;                       // event pairs used
    void reset()
    {
        for (int i = 0; i < PSCL_K_COUNT; i++) launches[i] = 0;
        n = 0;
    }
    void begin(cudaStream_t st)
    {
        if (ev && n < cap) cudaEventRecord(ev[2 * n], st);
    }
    void end(int k, cudaStream_t st)
    {
        launches[k]++;
        if (ev && n < cap) {
            cudaEventRecord(ev[2 * n + 1], st);
            tag[n++] = k;
        }
    }
};

// ---------------------------------------------------------------------- launchers
// All launchers queue work on `st` and return cudaGetLastError().

// scale.cu
// bf16: round the scaled values to bfloat16 (kept in float32).
cudaError_t launch_scale(const float *raw, float *x, int64_t n, int d, float *part,
                         uint32_t *ticket, double *mn, double *mx, uint32_t *flags, int sm_count,
                         cudaStream_t st, KTimer *kt, int bf16 = 0);
// bfloat16 points (bit patterns) widened to float32.
cudaError_t launch_widen_bf16(const uint16_t *in, float *out, int64_t count, int sm_count, cudaStream_t st);
size_t scale_part_floats(int64_t n, int d, int sm_count);
// Column minima / maxima of x (n x d) into mn / mx (part, ticket: as for launch_scale).
cudaError_t launch_minmax(const float *x, int64_t n, int d, float *part, uint32_t *ticket, double *mn, double *mx,
                          uint32_t *flags, int sm_count, cudaStream_t st, KTimer *kt);
// Independent sets: every set min-max scaled on its own (part: 2 x n_units x d floats,
// mn / mx: n_seg x d).
cudaError_t launch_seg_scale(const float *raw, float *x, const SegTable &t, const int32_t *seg_unit0, int d,
                             float *part, double *mn, double *mx, uint32_t *flags, cudaStream_t st, KTimer *kt);

// peel.cu
struct PeelBuffers {
    const float *x;                  // n x d scaled points
    uint32_t *rnd;                   // n: round (subcluster) of each point, all ones while unassigned
    uint8_t *pflag;                  // 2 x n: per CTA slice, a state byte per list position
    uint32_t *ord;                   // d x ord_ld: point ids of each attribute in bucket order
    uint32_t *bcnt;                  // d x nbuckets: bucket counts, then scatter cursors
    uint4 *bcs;                      // d x nbuckets: (points left, first entry, end entry, 0)
    uint32_t *lidx;                  // 2 x n: per CTA slice, the ids of its points left (two lists)
    uint32_t *kpos;                  // 2 x n: per CTA slice, the keys of its points left by list position
    int64_t ord_ld;                  // n rounded up to a multiple of 4
    uint32_t nbuckets;               // power of two, 4096 .. 65536
    uint32_t *band_k32;              // n: float32 keys of the epoch's band entries
    uint32_t *band_pos;              // n: their point ids
    uint64_t *gkey;                  // n: band entries regrouped by group (compensated distances)
    uint32_t *gpos;                  //    and their ids; the counting sort's second buffer afterwards
    uint64_t *akey;                  // n: entries near a group's cut-off (float64 distances)
    uint32_t *apos;                  //    and their ids
    uint32_t *pcnt;                  // 256 x perm_grid(n): counting-sort counts
    float *landmarks;                // all landmarks (S x d), for inspection
    uint32_t *perm;                  // n: subcluster-packed original indices
    float *xseg;                     // n x d: subcluster-packed points
    PeelCtl *ctl;
    uint32_t *flags;
    int rounds_per_pass;             // rounds one distance pass may serve (1..kMaxEpoch; 0: default)
    uint32_t wait_limit;             // polls of a bounded wait before it gives up (0: default)
    int stall_first_barrier;         // test hook: the first grid barrier waits for one CTA too many
    int max_grid = 0;                // most CTAs of the launch (0: as many as fit)
};
// Time per grid-wide barrier of the peel's own implementation, in the peel's launch shape
// (pscl_measure_grid_barrier).
cudaError_t measure_grid_barrier(int sm_count, double *us, bool *timed_out);
// Buckets of the per-attribute orders the peel builds for n points.
uint32_t peel_buckets(int64_t n);
// CTAs of the counting sort that packs the subclusters after the peel (pcnt: 256 x this).
int perm_grid(int64_t n, int sm_count);
// Rows of x in the order of perm, packed into xseg (the gather after any subclustering).
cudaError_t launch_gather(const float *x, const uint32_t *perm, int64_t n, int d, float *xseg, int sm_count,
                          cudaStream_t st, KTimer *kt);

// group.cu: Algorithm 2.  Landmarks lm (m x d) from lo / hi (the attributes' lowest and
// highest values), the group of every point, and perm = the points grouped in landmark
// order (ascending index inside a group); total[m] = each group's size.  cnt holds
// group_cnt_words(n, m) words.
constexpr int kMaxLandmarks = 4096;
size_t group_cnt_words(int64_t n, int m);
cudaError_t launch_group_unequal(const float *x, int64_t n, int d, const double *lo, const double *hi, int m,
                                 float *lm, int32_t *group, uint32_t *cnt, uint32_t *total, uint32_t *perm,
                                 cudaStream_t st, KTimer *kt);
// api.cu: route a job's peel through stream s (ordered with the job's own stream);
// a context's stream and device.
int job_set_coop_stream(pscl_job *j, cudaStream_t s);
cudaStream_t ctx_stream(const pscl_ctx *c);
int ctx_device(const pscl_ctx *c);

cudaError_t launch_peel(const PeelBuffers &b, int64_t n, int d, int64_t N, int sm_count,
                        cudaStream_t st, KTimer *kt);

// lloyd.cu
struct LloydBuffers {
    const float *pts;                // rows of all segments, packed
    float *centers;                  // P x d
    unsigned long long *acc;         // P x d fixed-point sums
    int32_t *count;                  // P counts of the current iteration (init: 2P, both)
    int32_t *labels;                 // rows
    int32_t *trace;                  // iters x rows (or NULL)
    int64_t rows;
    // rows' non-negative integer weights (or NULL: every weight 1).  A weighted row adds
    // w x to its center's sum and w to its count; such runs use the float32 assignment
    // with global 64-bit sums (w q needs up to 63 bits).
    const int32_t *weights = nullptr;
    // 8 words per row (or NULL): the tensor-core assignment marks a near tie's candidate
    // centers here (bit j of word j / 32), the sums pass re-scores only those
    uint32_t *tmask = nullptr;
    // a single set of more than 256 centers on the tensor cores: the rows as one set of 256
    // and of the remaining centers, with CTA splits (has_chunks), and 4 rows + 1 words of
    // scratch for the chunked search
    SegTable chunk256{}, chunkrem{};
    bool has_chunks = false;
    uint32_t *chunk_scratch = nullptr;
    uint32_t wait_limit = 0;         // polls of the tensor-core kernel's bounded waits (0: default)
    int tc_stall = 0;                // test hook: the tensor-core kernel waits once on a barrier nothing completes
};
cudaError_t launch_lloyd_init(const LloydBuffers &b, const SegTable &t, int d, int64_t P,
                              uint64_t seed, uint32_t stage, int first_k, int kmax,
                              cudaStream_t st, KTimer *kt);
// prec: a pscl_prec; TF32/BF16 use the tensor-core assignment where tc_supported() and the
// rows are unweighted.
cudaError_t launch_lloyd_iter(const LloydBuffers &b, int32_t *count_next, const SegTable &t,
                              int d, int iter, int unit_lo, int unit_hi, int64_t cen_lo,
                              int64_t cen_hi, int kmax, int prec, uint32_t *flags, int sm_count,
                              cudaStream_t st, KTimer *kt, int rows_per_thread = 0);
// Independent sets: nearest center of every row within its set, per-set sums of the
// squared distances (unit_sse: n_units doubles, seg_sse: n_seg doubles).
cudaError_t launch_seg_sse(const float *pts, const SegTable &t, const int32_t *seg_unit0, int d,
                           const float *centers, int kmax, int32_t *labels, double *unit_sse, double *seg_sse,
                           cudaStream_t st, KTimer *kt);

// lloyd_tc.cu
bool tc_supported(int d, int kmax, int prec);
// The SSE pass (labels and sum as launch_final_sse gives them) on the tensor cores for k
// centers in chunks of up to 256.  t256 / trem: the n rows as one set of 256 centers and of
// the k mod 256 remaining ones (k itself when k <= 256), with CTA splits; scratch: 4 n + 1
// words (row state and the list of rows re-scored in float32).
bool tc_sse_supported(int d, int k, int prec);
// One Lloyd iteration of a single set of k > 256 centers on the tensor cores (b.has_chunks):
// labels by the chunked search, then the exact sums; the update is launched separately.
cudaError_t launch_lloyd_chunks_tc(const LloydBuffers &b, int d, int iter, int k, int prec, uint32_t *flags,
                                   int sm_count, cudaStream_t st, KTimer *kt);
cudaError_t launch_final_sse_tc(const float *x, int64_t n, int d, const float *centers, int k, const SegTable &t256,
                                const SegTable &trem, uint32_t *scratch, int32_t *labels, double *blk_sse,
                                double *sse, uint32_t *ticket, int prec, uint32_t *flags, unsigned wait_limit,
                                int sm_count, cudaStream_t st, KTimer *kt);
// Assignment on the tensor cores and the exact sums of the iteration (two persistent
// launches over all units; needs t.split).
cudaError_t launch_lloyd_assign_tc(const LloydBuffers &b, const SegTable &t, int d, int iter, int kmax, int prec,
                                   uint32_t *flags, int sm_count, cudaStream_t st, KTimer *kt);
cudaError_t launch_final_sse(const float *x, int64_t n, int d, const float *centers, int k,
                             int32_t *labels, double *blk_sse, double *sse, uint32_t *ticket,
                             int sm_count, cudaStream_t st, KTimer *kt);
int sse_grid(int64_t n, int sm_count);

// api.cu: the message pscl_last_error() returns for the calling thread.
void set_last_error(const char *msg);

}  // namespace pscl
