// C ABI of the SGM path (include/sgm.h): context, device work arena, launch
// sequence and CUDA-graph cache, batched and served execution.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "sgm.h"
#include "sgm_check.cuh"
#include "sgm_internal.h"

using namespace sgm;

namespace sgm {
// The fault words of the bounds-checked build (sgm_check.cuh): one reader per
// translation unit, registered at load time.
static std::vector<unsigned (*)()>& bounds_readers() {
    static std::vector<unsigned (*)()> readers;
    return readers;
}
void register_bounds_reader(unsigned (*reader)()) { bounds_readers().push_back(reader); }
unsigned take_bounds_fault() {
    unsigned first = 0;
    for (auto reader : bounds_readers()) {
        const unsigned site = reader();
        if (site != 0 && first == 0) first = site;
    }
    return first;
}
// sgm_stages.cu: copy n bytes src0 -> dst0 and, when src1 is not null,
// src1 -> dst1 (pinned host buffers to or from the work arena).
cudaError_t launch_stage(const uint8_t* src0, uint8_t* dst0, const uint8_t* src1, uint8_t* dst1, size_t n,
                         cudaStream_t stream);
}  // namespace sgm

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Offsets of one pair's buffers inside a work arena.
struct Layout {
    size_t Fb, Fm, rec, raw, state, in_left, in_right, out, total;
    size_t sub, rawR, ml, mr;  // post-filters (sgm_compute_ex) only
    int RB;    // bytes per pixel record (sgm_internal.h): MC, S (room for u16 words), stored L_r fields;
               // the paired-line schedule: bytes of one quad in a cube (4D)
    int n_lx;  // stored-L_r fields per record
    size_t fs = 0;  // the paired-line schedule: bytes of one cube array
};

// Stored-L_r fields: one per pair of opposite paths whose first halves run
// concurrently (the horizontal pair and every vertical-type pair); none in
// 2-path mode.  Batched execution runs each pair's phases in one launch, one
// pair after the other, so a batched pair needs a single field and no phase
// state.
int lx_fields(int n_paths, bool batched) { return n_paths == 2 ? 0 : (batched ? 1 : (n_paths == 8 ? 4 : 2)); }

Layout layout_for(int W, int H, int D_int, int n_paths, bool batched = false, bool ct62 = false, bool post = false) {
    const size_t wh = static_cast<size_t>(W) * H;
    const size_t D = static_cast<size_t>(D_int);
    const size_t fbytes = ct62 ? 8 : 4;
    Layout l{};
    l.n_lx = lx_fields(n_paths, batched);
    l.RB = record_bytes(D_int, false, l.n_lx);
    size_t o = 0;
    l.Fb = o;  // features: uint32 (CSCT) or uint64 (full Census)
    o = align_up(o + fbytes * wh);
    l.Fm = o;
    o = align_up(o + fbytes * wh);
    l.rec = o;
    o = align_up(o + wh * static_cast<size_t>(l.RB));
    l.raw = o;
    o = align_up(o + wh);
    l.state = o;  // path states between the two phases of a pair: the vertical-type pairs (8 paths), the
                  // horizontal pair (4 paths)
    o = align_up(o + 4 * (n_paths == 8 ? 3 * sweep_state_words(W, static_cast<int>(D))
                                       : sweep_state_words(std::max(W, H), static_cast<int>(D))));
    l.in_left = o;
    o = align_up(o + wh);
    l.in_right = o;
    o = align_up(o + wh);
    l.out = o;
    o = align_up(o + (post ? 2 : 1) * wh);  // u16 output with post-filters
    if (post) {
        l.sub = o;  // per pixel S(d-1) - S(d) | (S(d+1) - S(d)) << 16 at the winner
        o = align_up(o + 4 * wh);
        l.rawR = o;  // the right pass's disparity, mirrored columns
        o = align_up(o + wh);
        l.ml = o;  // mirrored left and right images
        o = align_up(o + wh);
        l.mr = o;
        o = align_up(o + wh);
    }
    l.total = o;
    return l;
}

struct Problem {
    int W, H, D, P1, P2, n_paths;
    int ct62 = 0;  // features: 0 = CSCT (Eq. 1), 1 = the full 9x7 Census (SGM_FLAG_CENSUS_FULL)
    int post = 0;  // 0: the plain path (u8 output); else kPostOut16 | the SGM_POST_* flags of sgm_compute_ex
    int sched = 0;  // 4-path sweep schedule (SGM_SCHED_*)
    int n1 = -1;    // SGM_SCHED_PAIRS: horizontal steps in the first launch (-1: the default)
    int check_shrink = 0;  // bounds-checked build, test hook (PairsArgs::check_shrink)
};

// Set on every sgm_compute_ex problem: the post form with uint16 output, even
// without post-filters.
constexpr int kPostOut16 = 0x100;

// Largest matching cost: 31 CSCT bits or 62 full-Census bits.
inline int mc_max(const Problem& p) { return p.ct62 ? 62 : 31; }

// Largest jump penalty of a step: P2, or max(P1, P2) with adaptive P2.
inline int p2_max(const Problem& p) { return (p.post & SGM_POST_ADAPTIVE_P2) ? std::max(p.P1, p.P2) : p.P2; }

// S kept as bytes between the sweeps (sum_fits_u8 for this problem).
inline bool s8_for(const Problem& p) { return sum_fits_u8(p.n_paths, p2_max(p), mc_max(p)); }

// The paired-line schedule (SGM_SCHED_PAIRS) of a 4-path plain problem.
inline bool pairs_sched(const Problem& p) { return p.n_paths == 4 && !p.post && p.sched == SGM_SCHED_PAIRS; }

// Its 32-bit quad offsets (q * 4D) must stay below 4 GiB.
inline bool pairs_fit(const Problem& p) {
    const double W2 = p.W + (p.W & 1), H2 = p.H + (p.H & 1);
    return W2 * H2 * p.D < 4294967296.0;
}

// The quad cubes (one array of FS bytes per field), the quad raw disparity
// and the horizontal chains' state (sgm_internal.h); `RB` holds the bytes of
// one quad in a field (4D).
Layout layout_pairs(const Problem& p) {
    const PairsArgs g = pairs_geometry(p.W, p.H, p.D, p.n1);
    const size_t wh = static_cast<size_t>(p.W) * p.H, quads = static_cast<size_t>(g.QW) * g.QH;
    const size_t fbytes = p.ct62 ? 8 : 4;
    Layout l{};
    l.RB = 4 * p.D;
    l.fs = align_up(quads * static_cast<size_t>(l.RB));
    l.n_lx = 0;
    size_t o = 0;
    l.Fb = o;
    o = align_up(o + fbytes * wh);
    l.Fm = o;
    o = align_up(o + fbytes * wh);
    l.rec = o;
    o = align_up(o + kPairsFields * l.fs);
    l.raw = o;
    o = align_up(o + 4 * quads);
    l.state = o;
    o = align_up(o + 4 * static_cast<size_t>(g.QH) * 2 * 32 * (p.D / 32 + 1));
    l.in_left = o;
    o = align_up(o + wh);
    l.in_right = o;
    o = align_up(o + wh);
    l.out = o;
    o = align_up(o + wh);
    l.total = o;
    return l;
}

Layout schedule_layout(const Problem& p, bool batched) {
    if (!batched && pairs_sched(p)) return layout_pairs(p);
    return layout_for(p.W, p.H, p.D, p.n_paths, batched, p.ct62 != 0, p.post != 0);
}

// A 4-path plain problem may run any schedule (the tuner tries each on the
// same staged inputs): its staging buffers (in_left, in_right, out) sit past
// the working region of every schedule, so one arena serves them all.
Layout layout_for(const Problem& p, bool batched = false) {
    Layout l = schedule_layout(p, batched);
    if (batched || p.n_paths != 4 || p.post) return l;
    size_t base = 0;
    for (int s = 0; s <= SGM_SCHED_PAIRS; ++s) {
        Problem q = p;
        q.sched = s;
        if (s == SGM_SCHED_PAIRS && !pairs_fit(q)) continue;
        base = std::max(base, schedule_layout(q, false).in_left);
    }
    const size_t wh = static_cast<size_t>(p.W) * p.H;
    l.in_left = base;
    l.in_right = align_up(base + wh);
    l.out = align_up(l.in_right + wh);
    l.total = align_up(l.out + wh);
    return l;
}

size_t arena_need(const Problem& p) { return layout_for(p).total; }

bool valid_problem(const Problem& p, std::string* why) {
    char buf[160];
    if (p.W < 1 || p.H < 1) {
        snprintf(buf, sizeof buf, "W and H must be >= 1 (got %d x %d)", p.W, p.H);
    } else if (!supported_D(p.D)) {
        snprintf(buf, sizeof buf, "D must be a multiple of 32 in [32, %d] (got %d)", SGM_MAX_D, p.D);
    } else if (p.P1 < 0 || p.P1 > SGM_MAX_PENALTY || p.P2 < 0 || p.P2 > SGM_MAX_PENALTY) {
        snprintf(buf, sizeof buf, "P1 and P2 must lie in [0, %d] (got %d, %d)", SGM_MAX_PENALTY, p.P1, p.P2);
    } else if (p.ct62 && p.P2 > 255 - 62) {
        snprintf(buf, sizeof buf, "with the full Census P2 must lie in [0, %d] so that path costs fit a byte (got %d)",
                 255 - 62, p.P2);
    } else if (p.n_paths != 2 && p.n_paths != 4 && p.n_paths != 8) {
        snprintf(buf, sizeof buf, "n_paths must be 2, 4 or 8 (got %d)", p.n_paths);
    } else if (p.post & ~(kPostOut16 | SGM_POST_SUBPIXEL | SGM_POST_LR_CHECK | SGM_POST_ADAPTIVE_P2)) {
        snprintf(buf, sizeof buf, "unknown post-filter flags %#x", static_cast<unsigned>(p.post & ~kPostOut16));
    } else if ((p.post & SGM_POST_ADAPTIVE_P2) && p2_max(p) > 255 - mc_max(p)) {
        snprintf(buf, sizeof buf, "with adaptive P2, max(P1, P2) must not exceed %d (got %d)", 255 - mc_max(p),
                 p2_max(p));
    } else if (static_cast<double>(p.W) * p.H * record_bytes(p.D, false, lx_fields(p.n_paths, false)) >= 4294967296.0) {
        snprintf(buf, sizeof buf, "W*H*D too large (%d x %d x %d): the per-pixel records must stay below 4 GiB", p.W,
                 p.H, p.D);
    } else {
        return true;
    }
    *why = buf;
    return false;
}

struct GraphKey {
    Problem p;
    const void *left, *right, *out, *arena;
    bool operator<(const GraphKey& o) const {
        return std::tie(p.W, p.H, p.D, p.P1, p.P2, p.n_paths, p.ct62, p.post, p.sched, p.n1, left, right, out, arena) <
               std::tie(o.p.W, o.p.H, o.p.D, o.p.P1, o.p.P2, o.p.n_paths, o.p.ct62, o.p.post, o.p.sched, o.p.n1, o.left,
                        o.right, o.out, o.arena);
    }
};

struct Request {
    uint64_t ticket;
    Problem p;
    const uint8_t *left, *right;
    uint8_t* out;
    std::chrono::steady_clock::time_point t_submit;
};

// ---------------------------------------------------------------------------
// Batched execution state of one stream (sgm_compute_batch, or one served
// slot).  A wave of pairs is grouped by (D, path count, sum width, Census
// type); every stage of a group is one persistent grid over a device work
// list (sgm_internal.h).  The lists of a wave live in one blob: its pinned
// host image is filled per wave and copied to the device copy before the
// wave's graph runs.  The graph, captured once per wave shape (the groups'
// keys and the sweep grid) and replayed for every wave of that shape, zeroes
// the lists' counters, runs each group's stages on one of kListBranches
// concurrent branches, and copies the device status word back to the host.
// Blob layout: status word at 0, the counters at kBlobCounters, the WorkList
// headers at kBlobLists, the descriptors and prefix sums from kBlobHead.
// ---------------------------------------------------------------------------
constexpr int kListGroups = 16, kListBranches = 4, kListStages = 5, kListCounters = 8;
constexpr size_t kBlobCounters = 64, kBlobLists = 1024, kBlobListStride = 32, kBlobHead = 4096;
static_assert(kBlobCounters + 4 * kListGroups * kListCounters <= kBlobLists, "blob counters");
static_assert(kBlobLists + kBlobListStride * kListGroups * kListStages <= kBlobHead, "blob list headers");
static_assert(sizeof(WorkList<SweepArgs>) <= kBlobListStride, "work list header");
// Persistent blocks per SM of the sweep kernels the autotuner chooses among.
constexpr int kSweepGrids[] = {2, 3, 4, 5};
constexpr int kDefaultSweepGrid = 4;

struct ListExec {
    cudaStream_t capture = nullptr;
    cudaStream_t branch[kListBranches] = {};
    cudaEvent_t fork = nullptr, join[kListBranches] = {};
    uint8_t* blob_dev = nullptr;
    uint8_t* blob_host = nullptr;     // pinned, blob_cap bytes
    size_t blob_cap = 0;
    uint32_t* status_host = nullptr;  // pinned: the status word after the last wave
    std::map<std::pair<std::vector<int>, int>, cudaGraphExec_t> graphs;  // (group keys, sweep grid) -> graph
};

// Served execution: up to kServeSlots batches in flight, each on its own
// stream with its own arena from a device-resident pool.
constexpr int kServeSlots = 2;
constexpr int kServeMaxPairs = 64;

struct ServeSlot {
    sgm_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    uint8_t* arena = nullptr;
    size_t arena_bytes = 0;
    std::vector<Request> reqs;  // the batch in flight
    // pinned host staging for pageable inputs and outputs, so that no copy
    // blocks the scheduler; outputs are copied to the caller at retirement
    uint8_t* pinned = nullptr;
    size_t pinned_bytes = 0;
    std::vector<std::tuple<uint8_t*, const uint8_t*, size_t>> out_copies;
    ListExec exec;
    bool busy = false;          // reserved by the scheduler or running
    bool finished = false;      // set by the stream callback after the batch's last copy
    std::chrono::steady_clock::time_point t_done;
};

}  // namespace

struct sgm_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    // a second stream and two events that fork and join two kernels of one
    // path (the paired schedule's second launch), in and outside graph capture
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    size_t mem_cap = 0;
    uint8_t* arena = nullptr;
    size_t arena_bytes = 0;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::string err;
    std::atomic<uint64_t> launches{0};
    bool stage_timing = false;
    int ct62 = 0;  // SGM_FLAG_CENSUS_FULL
    cudaEvent_t stage_ev[10] = {};
    int last_stages = 0;
    int last_n_paths = 0;  // path count of the last path enqueued with stage timing
    int last_sched = 0;    // its sweep schedule
    // 4-path schedule: forced (>= 0) or autotuned per key (-1)
    int forced_sched = -1;
    std::map<std::tuple<int, int, int, int, int, bool>, int> tuned;  // (W, H, D, n_paths, ct62, s8) -> schedule
    cudaEvent_t tune_ev[2] = {};
    // batched execution: the caller's stream's list state, the SM count, the
    // sweep grid tuned per wave (its pairs' (W, H, D, n_paths), sorted)
    ListExec batch_exec;
    int n_sm = 0;
    std::map<std::vector<int>, int> list_tuned;

    // test hooks, read at sgm_create: SGM_TEST_FAIL_ALLOC=n fails the n-th
    // allocation; SGM_TEST_BAD_JOB=n gives n waves one descriptor with a D its
    // kernel rejects (through the device status word)
    int fail_alloc_at = 0;
    std::atomic<int> alloc_count{0};
    // bounds-checked build: SGM_TEST_BOUNDS_SHRINK=1 declares the paired
    // schedule's cube arrays one quad shorter than they are, so that a guard
    // fires on an access that is in fact in range
    bool bounds_shrink = false;
    std::atomic<int> bad_job_waves{0};

    // served requests
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, int> done;  // ticket -> status, finished and not yet polled
    std::unordered_set<uint64_t> outstanding;  // submitted and not yet retired by sgm_poll
    std::vector<double> latencies_us;
    uint64_t next_ticket = 1;
    size_t pending = 0;
    bool stop = false;
    bool worker_started = false;
    std::thread worker;
    ServeSlot slots[kServeSlots];
    std::atomic<size_t> serve_bytes{0};  // sum of the slots' arenas
    cudaMemPool_t serve_pool = nullptr;
    uint64_t batches = 0, batched_pairs = 0;
    int in_flight = 0, max_in_flight = 0;
    double served_de = 0.0;
    // admission bound (sgm_set_admission_bound): the backlog's disparity
    // evaluations over the measured service rate (all evaluations served over
    // the time with a batch in flight) estimate a new request's wait
    int64_t admit_max_us = 0;
    double backlog_de = 0.0, lifetime_de = 0.0, busy_us = 0.0;
    std::chrono::steady_clock::time_point busy_since;
    uint64_t shed = 0;
};

static thread_local std::string g_noctx_err;

static int fail(sgm_ctx* ctx, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_noctx_err = buf;
    return code;
}

#define CUDA_TRY(ctx, call)                                                                                   \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess)                                                                                \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? SGM_ENOMEM : SGM_ECUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                          \
    } while (0)

// Every device or pinned-host allocation of a context asks here first: the
// test hook SGM_TEST_FAIL_ALLOC=n makes the context's n-th allocation fail as
// if the device were out of memory, allocating nothing.
static bool injected_alloc_failure(sgm_ctx* ctx) {
    return ctx->fail_alloc_at > 0 && ctx->alloc_count.fetch_add(1) + 1 == ctx->fail_alloc_at;
}

static cudaError_t ctx_malloc(sgm_ctx* ctx, void** p, size_t bytes) {
    return injected_alloc_failure(ctx) ? cudaErrorMemoryAllocation : cudaMalloc(p, bytes);
}

static cudaError_t ctx_malloc_host(sgm_ctx* ctx, void** p, size_t bytes) {
    return injected_alloc_failure(ctx) ? cudaErrorMemoryAllocation : cudaMallocHost(p, bytes);
}

// After a synchronous call in the bounds-checked build: SGM_EDEVICE if a
// kernel's guard fired (sgm_check.cuh).  Always SGM_OK in the ordinary build.
static int bounds_status(sgm_ctx* ctx) {
#ifdef SGM_BOUNDS_CHECK
    const unsigned site = take_bounds_fault();
    if (site != 0) return fail(ctx, SGM_EDEVICE, "bounds check: an access out of its array at site %u", site);
#else
    (void)ctx;
#endif
    return SGM_OK;
}

static int ensure_arena(sgm_ctx* ctx, uint8_t** arena, size_t* bytes, size_t need, bool clear_graphs) {
    if (*bytes >= need) return SGM_OK;
    const size_t used_elsewhere = ctx->serve_bytes.load();
    if (ctx->mem_cap && need + used_elsewhere > ctx->mem_cap)
        return fail(ctx, SGM_ENOMEM, "work arena of %zu bytes exceeds the context's memory cap of %zu bytes", need,
                    ctx->mem_cap);
    if (*arena) {
        cudaError_t e = cudaFree(*arena);
        *arena = nullptr;
        *bytes = 0;
        if (e != cudaSuccess) return fail(ctx, SGM_ECUDA, "cudaFree: %s", cudaGetErrorString(e));
    }
    if (clear_graphs) {
        for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
        ctx->graphs.clear();
    }
    void* p = nullptr;
    cudaError_t e = ctx_malloc(ctx, &p, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SGM_ENOMEM, "cudaMalloc(%zu) for the work arena: %s", need, cudaGetErrorString(e));
    }
    *arena = static_cast<uint8_t*>(p);
    *bytes = need;
    return SGM_OK;
}

static cudaMemoryType pointer_kind(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return cudaMemoryTypeUnregistered;
    }
    return at.type;
}

static bool is_device_ptr(const void* p) {
    const cudaMemoryType t = pointer_kind(p);
    return t == cudaMemoryTypeDevice || t == cudaMemoryTypeManaged;
}

// Kernels per path: census, cost, the first sweep stage (horizontal pair and
// vertical-type first halves), the second halves of each vertical-type pair
// (sweep_diag+, sweep_diag-, sweep_v), median; with 2 paths: census, cost,
// sweep_h, sweep_v, median.  Each kernel is one timed stage.  With
// post-filters: one matching pass (census, cost, sweeps) for the left image,
// with the LR check a mirror kernel and a second pass, then the post kernel.
// The paired schedule runs its second launch as two kernels side by side (one
// timed stage).
static int launches_per_match(const Problem& p) { return p.n_paths == 8 ? 6 : (pairs_sched(p) ? 5 : 4); }
static int launches_per_path(const Problem& p) {
    if (!p.post) return launches_per_match(p) + 1;
    return launches_per_match(p) * ((p.post & SGM_POST_LR_CHECK) ? 2 : 1) + ((p.post & SGM_POST_LR_CHECK) ? 1 : 0) + 1;
}
static int stages_per_path(const Problem& p) { return launches_per_path(p) - (pairs_sched(p) ? 1 : 0); }

// Two kernels of one path side by side: `aux` waits for `fork` recorded on
// the path's stream, the path's stream waits for `join` recorded on `aux`.
struct ForkJoin {
    cudaStream_t aux;
    cudaEvent_t fork, join;
};

// One matching pass (Section 2, stages 2-3 and Eq. 4) of the pair
// (base, match): census, cost and the sweeps; the winner-take-all disparity
// goes to raw.  In the post form the sweeps take their jump penalties from
// base's intensities and, with sub, write the winner's neighbour sums.
template <class Mark>
static cudaError_t enqueue_match(const Problem& p, const Layout& l, uint8_t* arena, const uint8_t* base,
                                 const uint8_t* match, uint8_t* raw, uint32_t* sub, uint16_t* Sdbg, cudaStream_t s,
                                 const ForkJoin& fj, Mark&& mark) {
    void* Fb = arena + l.Fb;
    void* Fm = arena + l.Fm;
    cudaError_t e;
    if ((e = launch_census(base, match, Fb, Fm, p.W, p.H, p.ct62 != 0, s)) != cudaSuccess) return e;
    if ((e = mark()) != cudaSuccess) return e;
    if (pairs_sched(p)) {
        // two lines per warp over quad cubes: the costs, then every walker
        // storing its L_r beside the others, then the horizontal rest with
        // Eq. 4 beside the parallel winner-take-all; raw in quads
        if ((e = launch_cost_quads(Fb, Fm, arena + l.rec, l.RB, p.W, p.H, p.D, p.ct62 != 0, s)) != cudaSuccess)
            return e;
        if ((e = mark()) != cudaSuccess) return e;
        PairsArgs g = pairs_geometry(p.W, p.H, p.D, p.n1);
        g.rec = arena + l.rec;
        g.rawq = raw;
        g.Sdbg = Sdbg;
        g.state = reinterpret_cast<uint32_t*>(arena + l.state);
        g.QB = l.RB;
        g.FS = l.fs;
        g.P1x2 = static_cast<uint32_t>(p.P1) * 0x10001u;
        g.P2x2 = static_cast<uint32_t>(p.P2) * 0x10001u;
        g.s8 = s8_for(p) ? 1 : 0;
        g.mc_max = mc_max(p);
        g.check_shrink = p.check_shrink;
        if ((e = launch_pairs_stage1(g, s)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
        // the horizontal chains (the long pole: enqueued first) and the
        // parallel winner-take-all side by side
        if ((e = cudaEventRecord(fj.fork, s)) != cudaSuccess) return e;
        if ((e = launch_pairs_chain2(g, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(fj.aux, fj.fork, 0)) != cudaSuccess) return e;
        if ((e = launch_pairs_par(g, fj.aux)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(fj.join, fj.aux)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, fj.join, 0)) != cudaSuccess) return e;
        return mark();
    }
    if ((e = launch_cost(Fb, Fm, arena + l.rec, l.RB, p.W, p.H, p.D, p.ct62 != 0, s)) != cudaSuccess) return e;
    if ((e = mark()) != cudaSuccess) return e;
    SweepArgs a{};
    a.rec = arena + l.rec;
    a.RB = l.RB;
    a.lx_off = 3 * p.D;  // stored-L_r field k at 3D + kD: the horizontal pair takes field 0
    a.raw = raw;
    a.Sdbg = Sdbg;
    a.W = p.W;
    a.H = p.H;
    a.D = p.D;
    a.P1x2 = static_cast<uint32_t>(p.P1) * 0x10001u;
    a.P2x2 = static_cast<uint32_t>(p.P2) * 0x10001u;
    a.pair = p.n_paths >= 4;
    a.s8 = s8_for(p);
    a.rx = 0;
    a.wta = 0;
    a.phase = 0;
    a.post = p.post ? 1 : 0;
    a.img = base;
    a.ap2 = (p.post & SGM_POST_ADAPTIVE_P2) ? 1 : 0;
    a.sub = sub;
    uint32_t* states = reinterpret_cast<uint32_t*>(arena + l.state);
    const size_t sw = sweep_state_words(p.W, p.D);
    a.state_end = states + (p.n_paths == 8 ? 3 * sw : sweep_state_words(std::max(p.W, p.H), p.D));
    // vertical-type pairs: (rx, wta) in the order their second halves run
    const int nv = p.n_paths == 8 ? 3 : 1;
    const int vrx[3] = {1, -1, 0};
    const int* rxs = p.n_paths == 8 ? vrx : vrx + 2;
    if (!a.pair) {
        // 2-path mode: left-to-right, then top-to-bottom with the winner-take-all
        if ((e = launch_sweep_h(a, s)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
        a.wta = 1;
        if ((e = launch_sweep_v(a, s)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
    } else if (p.n_paths == 4 && p.sched == SGM_SCHED_H_THEN_V) {
        // 4 paths, the other schedule: the whole horizontal pair
        // (S = L_LR + L_RL) beside the vertical first halves, then the
        // vertical second halves with Eq. 4
        FirstStageArgs f{};
        f.h = a;
        f.nv = 1;
        f.v[0] = a;
        f.v[0].phase = 1;
        f.v[0].state = states;
        f.v[0].lx_off = 4 * p.D;
        if ((e = launch_sweep_first(f, s)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
        SweepArgs b = a;
        b.phase = 2;
        b.wta = 1;
        b.state = states;
        b.lx_off = 4 * p.D;
        if ((e = launch_sweep_v(b, s)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
    } else if (p.n_paths == 4) {
        // 4 paths: the whole vertical pair (S = L_TB + L_BT) beside the
        // horizontal first halves, then the horizontal second halves with Eq. 4
        FirstStageArgs f{};
        f.h = a;
        f.h.state = states;
        f.nv = 1;
        f.v[0] = a;
        f.v[0].lx_off = 4 * p.D;  // the vertical pair's stored-L_r field
        if ((e = launch_sweep_first4(f, s)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
        SweepArgs b = a;
        b.state = states;
        b.wta = 1;
        b.phase = 2;
        if ((e = launch_sweep_h2(b, s)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
    } else {
        // the first halves of the vertical-type pairs need only the costs: they
        // run in the same launch as the horizontal pair
        FirstStageArgs f{};
        f.h = a;
        f.nv = nv;
        for (int v = 0; v < nv; ++v) {
            SweepArgs b = a;
            b.rx = rxs[v];
            b.phase = 1;
            b.state = states + v * sw;
            // each vertical-type pair keeps its own stored-L_r field
            b.lx_off = (4 + v) * p.D;
            f.v[v] = b;
        }
        if ((e = launch_sweep_first(f, s)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
        for (int v = 0; v < nv; ++v) {
            SweepArgs b = a;
            b.rx = rxs[v];
            b.phase = 2;
            b.wta = (rxs[v] == 0) ? 1 : 0;
            b.state = states + v * sw;
            b.lx_off = (4 + v) * p.D;
            if ((e = launch_sweep_v(b, s)) != cudaSuccess) return e;
            if ((e = mark()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Enqueue the whole path (Section 2, stages 2-4) for one pair whose inputs
// and output are device pointers: disp is uint8 [H][W], or uint16 [H][W] in
// 1/16 pixel with post-filters (p.post).  Returns a cudaError_t.
static cudaError_t enqueue_path(sgm_ctx* ctx, const Problem& p, uint8_t* arena, const uint8_t* left,
                                const uint8_t* right, uint8_t* disp, uint16_t* Sdbg, cudaStream_t s, bool timed) {
    const Layout l = layout_for(p);
    const ForkJoin fj{ctx->aux_stream, ctx->fork_ev, ctx->join_ev};
    cudaError_t e;
    int stage = 0;
    // with stage timing, event k is recorded before kernel k and after the last
    auto mark = [&]() -> cudaError_t {
        if (!timed) return cudaSuccess;
        // External: inside a stream capture this becomes an event-record node of the graph
        return cudaEventRecordWithFlags(ctx->stage_ev[stage++], s, cudaEventRecordExternal);
    };
    if ((e = mark()) != cudaSuccess) return e;
    if (!p.post) {
        if ((e = enqueue_match(p, l, arena, left, right, arena + l.raw, nullptr, Sdbg, s, fj, mark)) != cudaSuccess)
            return e;
        e = pairs_sched(p) ? launch_median_quads(arena + l.raw, disp, p.W, p.H, s)
                           : launch_median(arena + l.raw, disp, p.W, p.H, s);
        if (e != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
    } else {
        uint32_t* sub = (p.post & SGM_POST_SUBPIXEL) ? reinterpret_cast<uint32_t*>(arena + l.sub) : nullptr;
        if ((e = enqueue_match(p, l, arena, left, right, arena + l.raw, sub, nullptr, s, fj, mark)) != cudaSuccess)
            return e;
        const uint8_t* rawR = nullptr;
        if (p.post & SGM_POST_LR_CHECK) {
            // the right image's disparity: the same pass on the mirrored pair
            if ((e = launch_mirror(left, right, arena + l.ml, arena + l.mr, p.W, p.H, s)) != cudaSuccess) return e;
            if ((e = mark()) != cudaSuccess) return e;
            if ((e = enqueue_match(p, l, arena, arena + l.mr, arena + l.ml, arena + l.rawR, nullptr, nullptr, s, fj,
                                   mark)) != cudaSuccess)
                return e;
            rawR = arena + l.rawR;
        }
        if ((e = launch_post(arena + l.raw, sub, rawR, reinterpret_cast<uint16_t*>(disp), p.W, p.H, p.D, s)) !=
            cudaSuccess)
            return e;
        if ((e = mark()) != cudaSuccess) return e;
    }
    ctx->launches += launches_per_path(p);
    return cudaSuccess;
}

// Pinned host buffers of one call, copied by staging kernels that are part of
// the call's graph: the images into the arena before the path, the output out
// of it after.
struct HostIO {
    const uint8_t* src[2] = {nullptr, nullptr};  // host images
    uint8_t* dst[2] = {nullptr, nullptr};        // their arena copies
    const uint8_t* out_src = nullptr;            // arena output
    uint8_t* out_dst = nullptr;                  // host output
    size_t img_bytes = 0, out_bytes = 0;
    int launches() const { return (src[0] ? 1 : 0) + (out_src ? 1 : 0); }
};

// Enqueue through a cached CUDA graph for this problem and these pointers.
// The key names the caller's buffers (a staged host buffer's arena copy is the
// same for every host buffer).  An address that is staged in one call and
// used in place in another (freed and reused as another kind of memory)
// reuses the first call's graph, which is correct for either kind: the copies
// work on device memory, and the kernels can read pinned host memory.
static int enqueue_graph(sgm_ctx* ctx, const Problem& p, uint8_t* arena, const uint8_t* left, const uint8_t* right,
                         uint8_t* disp, cudaStream_t s, const HostIO& io = HostIO{}, const void* key_left = nullptr,
                         const void* key_right = nullptr, const void* key_out = nullptr) {
    GraphKey key{p, key_left ? key_left : left, key_right ? key_right : right, key_out ? key_out : disp, arena};
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        if (ctx->graphs.size() >= 64) {
            for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
            ctx->graphs.clear();
        }
        cudaGraph_t g = nullptr;
        CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        const uint64_t before = ctx->launches.load();
        cudaError_t e = cudaSuccess;
        if (io.src[0]) e = launch_stage(io.src[0], io.dst[0], io.src[1], io.dst[1], io.img_bytes, ctx->capture_stream);
        // paths with post-filters are never stage-timed (sgm_stage_times names the plain path's kernels)
        if (e == cudaSuccess)
            e = enqueue_path(ctx, p, arena, left, right, disp, nullptr, ctx->capture_stream,
                             ctx->stage_timing && !p.post);
        if (e == cudaSuccess && io.out_src)
            e = launch_stage(io.out_src, io.out_dst, nullptr, nullptr, io.out_bytes, ctx->capture_stream);
        ctx->launches = before;  // captured, not launched
        cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(ctx, SGM_ECUDA, "graph capture failed: %s / %s", cudaGetErrorString(e),
                        cudaGetErrorString(e2));
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(ctx, SGM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        it = ctx->graphs.emplace(key, exec).first;
    }
    CUDA_TRY(ctx, cudaGraphLaunch(it->second, s));
    ctx->launches += launches_per_path(p) + io.launches();
    ctx->last_stages = (ctx->stage_timing && !p.post) ? stages_per_path(p) : 0;
    ctx->last_n_paths = (ctx->stage_timing && !p.post) ? p.n_paths : 0;
    ctx->last_sched = p.sched;
    return SGM_OK;
}

// The 4-path sweep schedule of a plain-path problem: forced, or the fastest of
// the kSchedules measured on the first use of its (W, H, D, Census, byte sums)
// key.  Tuning runs the whole path (into the caller's output, which every
// schedule computes bit-identically) once per schedule to warm up and
// kTuneReps times timed with events on `s`; the median decides.  A stream
// under capture cannot be timed: there the default schedule is used untuned.
constexpr int kSchedules = 3, kTuneReps = 5;
static int choose_schedule(sgm_ctx* ctx, Problem& p, uint8_t* arena, const uint8_t* left, const uint8_t* right,
                           uint8_t* disp, cudaStream_t s) {
    p.sched = SGM_SCHED_V_THEN_H;
    if (p.n_paths != 4 || p.post) return SGM_OK;
    if (ctx->forced_sched >= 0) {
        p.sched = ctx->forced_sched;
        if (pairs_sched(p) && !pairs_fit(p)) p.sched = SGM_SCHED_V_THEN_H;  // quad records would pass 4 GiB
        return SGM_OK;
    }
    const auto key = std::make_tuple(p.W, p.H, p.D, p.n_paths, p.ct62, s8_for(p));
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
        p.sched = it->second;
        return SGM_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_TRY(ctx, cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return SGM_OK;
    float best_ms = 0.f;
    int best = -1;
    for (int sched = 0; sched < kSchedules; ++sched) {
        Problem q = p;
        q.sched = sched;
        if (sched == SGM_SCHED_PAIRS && !pairs_fit(q)) continue;
        int rc = enqueue_graph(ctx, q, arena, left, right, disp, s);  // captures the graph; warm-up
        if (rc != SGM_OK) return rc;
        float ms[kTuneReps];
        for (int rep = 0; rep < kTuneReps; ++rep) {
            CUDA_TRY(ctx, cudaEventRecord(ctx->tune_ev[0], s));
            if ((rc = enqueue_graph(ctx, q, arena, left, right, disp, s)) != SGM_OK) return rc;
            CUDA_TRY(ctx, cudaEventRecord(ctx->tune_ev[1], s));
            CUDA_TRY(ctx, cudaEventSynchronize(ctx->tune_ev[1]));
            CUDA_TRY(ctx, cudaEventElapsedTime(&ms[rep], ctx->tune_ev[0], ctx->tune_ev[1]));
        }
        std::sort(ms, ms + kTuneReps);
        const float med = ms[kTuneReps / 2];
        if (best < 0 || med < best_ms) {
            best = sched;
            best_ms = med;
        }
    }
    p.sched = best;
    ctx->tuned.emplace(key, p.sched);
    return SGM_OK;
}

// Copy-in / path / copy-out for one pair into `arena` (already large enough).
// Device memory and pinned host memory are read and written in place by the
// kernels (pinned host memory is mapped into the device's address space, so
// the census reads the images and the last kernel writes the output over the
// host link with no separate copy); pageable host memory is staged through
// the arena with copies.
static int enqueue_pair(sgm_ctx* ctx, const Problem& p, uint8_t* arena, const uint8_t* left, const uint8_t* right,
                        uint8_t* disp, cudaStream_t s, bool use_graph) {
    const Layout l = layout_for(p);
    const size_t wh = static_cast<size_t>(p.W) * p.H;
    // device buffers are used in place; pinned host buffers are copied by
    // staging kernels (each byte crosses the host link once, in wide
    // requests; the Census tiles would read every image byte several times
    // over the link), inside the call's graph; pageable host buffers by
    // cudaMemcpyAsync before and after it
    const cudaMemoryType kl = pointer_kind(left), kr = pointer_kind(right), ko = pointer_kind(disp);
    auto device_side = [](cudaMemoryType t) { return t == cudaMemoryTypeDevice || t == cudaMemoryTypeManaged; };
    const uint8_t* dl = left;
    const uint8_t* dr = right;
    uint8_t* dout = disp;
    HostIO io;
    io.img_bytes = wh;
    int n_st = 0;
    if (!device_side(kl)) {
        dl = arena + l.in_left;
        if (kl == cudaMemoryTypeHost) {
            io.src[n_st] = left;
            io.dst[n_st++] = arena + l.in_left;
        } else {
            CUDA_TRY(ctx, cudaMemcpyAsync(arena + l.in_left, left, wh, cudaMemcpyHostToDevice, s));
        }
    }
    if (!device_side(kr)) {
        dr = arena + l.in_right;
        if (kr == cudaMemoryTypeHost) {
            io.src[n_st] = right;
            io.dst[n_st++] = arena + l.in_right;
        } else {
            CUDA_TRY(ctx, cudaMemcpyAsync(arena + l.in_right, right, wh, cudaMemcpyHostToDevice, s));
        }
    }
    const size_t ob = (p.post ? 2 : 1) * wh;
    if (!device_side(ko)) {
        dout = arena + l.out;
        if (ko == cudaMemoryTypeHost) {
            io.out_src = dout;
            io.out_dst = disp;
            io.out_bytes = ob;
        }
    }
    if (use_graph) {
        // the tuner's runs read the arena copies before this call's staging
        // has filled them: their timing does not depend on the values, and
        // the graph launched below recomputes the result from the staged ones
        Problem q = p;
        int rc = choose_schedule(ctx, q, arena, dl, dr, dout, s);
        if (rc != SGM_OK) return rc;
        rc = enqueue_graph(ctx, q, arena, dl, dr, dout, s, io, left, right, disp);
        if (rc != SGM_OK) return rc;
    } else {
        if (io.src[0]) CUDA_TRY(ctx, launch_stage(io.src[0], io.dst[0], io.src[1], io.dst[1], wh, s));
        CUDA_TRY(ctx, enqueue_path(ctx, p, arena, dl, dr, dout, nullptr, s, false));
        if (io.out_src) CUDA_TRY(ctx, launch_stage(io.out_src, io.out_dst, nullptr, nullptr, ob, s));
        ctx->launches += io.launches();
    }
    if (!device_side(ko) && ko != cudaMemoryTypeHost)
        CUDA_TRY(ctx, cudaMemcpyAsync(disp, dout, ob, cudaMemcpyDeviceToHost, s));
    return SGM_OK;
}

// A problem as the context sees it (its Census type).
static Problem make_problem(const sgm_ctx* ctx, int W, int H, int D, int P1, int P2, int n_paths) {
    Problem p{W, H, D, P1, P2, n_paths};
    p.ct62 = ctx ? ctx->ct62 : 0;
    p.check_shrink = (ctx && ctx->bounds_shrink) ? 4 * D : 0;
    return p;
}

static int check_args(sgm_ctx* ctx, const Problem& p, const void* left, const void* right, const void* out) {
    if (!ctx) return fail(nullptr, SGM_EINVAL, "null context");
    if (!left || !right || !out) return fail(ctx, SGM_EINVAL, "null image or output pointer");
    std::string why;
    if (!valid_problem(p, &why)) return fail(ctx, SGM_EINVAL, "%s", why.c_str());
    return SGM_OK;
}

// ---------------------------------------------------------------------------
// Batched execution: pairs grouped by (D, n_paths, sum width, Census type),
// each group's stages as persistent grids over device work lists, the whole
// wave one graph launch.  Pairs are packed into waves whose buffers fit the
// memory budget; each pair has its own region of the arena.
// ---------------------------------------------------------------------------
struct BatchItem {
    Problem p;
    const uint8_t *left, *right;
    uint8_t* out;
    size_t offset;  // of the pair's region in the arena
};

// Items of one group share D, the path count, the sum storage and the Census type.
static std::tuple<int, int, bool, int> batch_key(const BatchItem& it) {
    return std::make_tuple(it.p.D, it.p.n_paths, s8_for(it.p), it.p.ct62);
}

static int group_code(const BatchItem& it) {
    return it.p.D | it.p.n_paths << 9 | (s8_for(it.p) ? 1 : 0) << 13 | it.p.ct62 << 14;
}

static int launches_per_group(int n_paths) { return 4 + (n_paths == 8 ? 3 : 1); }

static int list_exec_init(sgm_ctx* ctx, ListExec& x) {
    CUDA_TRY(ctx, cudaStreamCreateWithFlags(&x.capture, cudaStreamNonBlocking));
    CUDA_TRY(ctx, cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming));
    for (int b = 0; b < kListBranches; ++b) {
        CUDA_TRY(ctx, cudaStreamCreateWithFlags(&x.branch[b], cudaStreamNonBlocking));
        CUDA_TRY(ctx, cudaEventCreateWithFlags(&x.join[b], cudaEventDisableTiming));
    }
    void* q = nullptr;
    CUDA_TRY(ctx, ctx_malloc_host(ctx, &q, sizeof(uint32_t)));
    x.status_host = static_cast<uint32_t*>(q);
    *x.status_host = 0;
    return SGM_OK;
}

static void list_exec_clear_graphs(ListExec& x) {
    for (auto& kv : x.graphs) cudaGraphExecDestroy(kv.second);
    x.graphs.clear();
}

static void list_exec_release(ListExec& x) {
    list_exec_clear_graphs(x);
    if (x.blob_dev) cudaFree(x.blob_dev);
    if (x.blob_host) cudaFreeHost(x.blob_host);
    if (x.status_host) cudaFreeHost(x.status_host);
    for (int b = 0; b < kListBranches; ++b) {
        if (x.branch[b]) cudaStreamDestroy(x.branch[b]);
        if (x.join[b]) cudaEventDestroy(x.join[b]);
    }
    if (x.fork) cudaEventDestroy(x.fork);
    if (x.capture) cudaStreamDestroy(x.capture);
    x = ListExec{};
}

// Room for `bytes` of blob (device copy and pinned host image); a new blob
// moves the lists, so the graphs that point into the old one go.
static int list_exec_reserve(sgm_ctx* ctx, ListExec& x, size_t bytes) {
    if (x.blob_cap >= bytes) return SGM_OK;
    const size_t cap = std::max(bytes, x.blob_cap * 2);
    list_exec_clear_graphs(x);
    if (x.blob_dev) CUDA_TRY(ctx, cudaFree(x.blob_dev));
    if (x.blob_host) CUDA_TRY(ctx, cudaFreeHost(x.blob_host));
    x.blob_dev = x.blob_host = nullptr;
    x.blob_cap = 0;
    void *d = nullptr, *h = nullptr;
    CUDA_TRY(ctx, ctx_malloc(ctx, &d, cap));
    x.blob_dev = static_cast<uint8_t*>(d);
    CUDA_TRY(ctx, ctx_malloc_host(ctx, &h, cap));
    x.blob_host = static_cast<uint8_t*>(h);
    x.blob_cap = cap;
    return SGM_OK;
}

// The groups of a wave: [first item, end) per group, at most kListGroups
// (items sorted by batch_key; a longer run of groups goes to the next wave).
static std::vector<std::pair<size_t, size_t>> wave_groups(const std::vector<BatchItem>& items, size_t b, size_t e) {
    std::vector<std::pair<size_t, size_t>> g;
    for (size_t g0 = b; g0 < e;) {
        size_t g1 = g0;
        while (g1 < e && batch_key(items[g1]) == batch_key(items[g0])) ++g1;
        g.emplace_back(g0, g1);
        g0 = g1;
    }
    return g;
}

// Fill the blob's host image with the lists of a wave's groups; returns its
// used bytes, or 0 with *rc set on failure.
static size_t build_lists(sgm_ctx* ctx, ListExec& x, const std::vector<BatchItem>& items,
                          const std::vector<std::pair<size_t, size_t>>& groups, uint8_t* arena, int* rc) {
    auto up8 = [](size_t v) { return (v + 7) & ~size_t(7); };
    size_t need = kBlobHead;
    for (const auto& g : groups) {
        const size_t n = g.second - g.first;
        need += up8(n * sizeof(CensusJob)) + up8(n * sizeof(CostJob)) + 2 * up8(n * sizeof(SweepArgs)) +
                up8(n * sizeof(MedianJob)) + kListStages * up8((n + 1) * sizeof(uint32_t));
    }
    if ((*rc = list_exec_reserve(ctx, x, need)) != SGM_OK) return 0;
    std::memset(x.blob_host, 0, kBlobHead);
    size_t off = kBlobHead;
    auto place = [&](const void* src, size_t bytes) -> const void* {
        const size_t o = off;
        std::memcpy(x.blob_host + o, src, bytes);
        off = up8(o + bytes);
        return x.blob_dev + o;
    };
    auto header = [&](size_t g, int stage, const void* job, const void* start, int n) {
        WorkList<CensusJob> w{static_cast<const CensusJob*>(job), static_cast<const uint32_t*>(start), n};
        std::memcpy(x.blob_host + kBlobLists + (g * kListStages + stage) * kBlobListStride, &w, sizeof w);
    };
    for (size_t g = 0; g < groups.size(); ++g) {
        const size_t g0 = groups[g].first, n = groups[g].second - g0;
        std::vector<CensusJob> cj(n);
        std::vector<CostJob> mj(n);
        std::vector<SweepArgs> hj, vj;
        std::vector<MedianJob> dj(n);
        std::vector<uint32_t> cs(n + 1, 0), ms(n + 1, 0), hs(n + 1, 0), vs(n + 1, 0), ds(n + 1, 0);
        std::vector<SweepArgs> sa(n);
        for (size_t k = 0; k < n; ++k) {
            const BatchItem& it = items[g0 + k];
            const Layout l = layout_for(it.p, true);
            uint8_t* base = arena + it.offset;
            void* Fb = base + l.Fb;
            void* Fm = base + l.Fm;
            cj[k] = CensusJob{it.left, it.right, Fb, Fm, it.p.W, it.p.H};
            mj[k] = CostJob{Fb, Fm, base + l.rec, l.RB, it.p.W, it.p.H, it.p.D};
            SweepArgs a{};
            a.rec = base + l.rec;
            a.RB = l.RB;
            a.lx_off = 3 * it.p.D;  // one stored-L_r field, reused pair after pair
            a.raw = base + l.raw;
            a.W = it.p.W;
            a.H = it.p.H;
            a.D = it.p.D;
            a.P1x2 = static_cast<uint32_t>(it.p.P1) * 0x10001u;
            a.P2x2 = static_cast<uint32_t>(it.p.P2) * 0x10001u;
            a.pair = it.p.n_paths >= 4;
            a.s8 = s8_for(it.p);
            sa[k] = a;
            uint8_t* dst = is_device_ptr(it.out) ? it.out : base + l.out;
            dj[k] = MedianJob{base + l.raw, dst, it.p.W, it.p.H};
            cs[k + 1] = cs[k] + census_units(it.p.W, it.p.H);
            ms[k + 1] = ms[k] + cost_units(it.p.W, it.p.H);
            ds[k + 1] = ds[k] + median_units(it.p.W, it.p.H);
        }
        // the sweeps hand out the longest chains first: rows by width, columns by height
        std::vector<size_t> oh(n), ov(n);
        for (size_t k = 0; k < n; ++k) oh[k] = ov[k] = k;
        std::stable_sort(oh.begin(), oh.end(), [&](size_t i, size_t j) { return sa[i].W > sa[j].W; });
        std::stable_sort(ov.begin(), ov.end(), [&](size_t i, size_t j) { return sa[i].H > sa[j].H; });
        for (size_t k = 0; k < n; ++k) {
            hj.push_back(sa[oh[k]]);
            vj.push_back(sa[ov[k]]);
            hs[k + 1] = hs[k] + sweep_units(sa[oh[k]].H, sa[oh[k]].D, sa[oh[k]].pair);
            vs[k + 1] = vs[k] + sweep_units(sa[ov[k]].W, sa[ov[k]].D, sa[ov[k]].pair);
        }
        if (g == 0 && ctx->bad_job_waves.load() > 0) {  // test hook: a descriptor its kernel must reject
            --ctx->bad_job_waves;
            hj[0].D += 32;
        }
        const int ni = static_cast<int>(n);
        header(g, 0, place(cj.data(), n * sizeof(CensusJob)), place(cs.data(), (n + 1) * 4), ni);
        header(g, 1, place(mj.data(), n * sizeof(CostJob)), place(ms.data(), (n + 1) * 4), ni);
        header(g, 2, place(hj.data(), n * sizeof(SweepArgs)), place(hs.data(), (n + 1) * 4), ni);
        header(g, 3, place(vj.data(), n * sizeof(SweepArgs)), place(vs.data(), (n + 1) * 4), ni);
        header(g, 4, place(dj.data(), n * sizeof(MedianJob)), place(ds.data(), (n + 1) * 4), ni);
    }
    return off;
}

// The graph of a wave shape: counters zeroed, each group's stages on a
// branch, the status word copied back.
static int list_graph(sgm_ctx* ctx, ListExec& x, const std::vector<int>& keys, int sweep_grid,
                      cudaGraphExec_t* out) {
    const auto key = std::make_pair(keys, sweep_grid);
    auto it = x.graphs.find(key);
    if (it != x.graphs.end()) {
        *out = it->second;
        return SGM_OK;
    }
    cudaStream_t c = x.capture;
    CUDA_TRY(ctx, cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal));
    auto body = [&]() -> cudaError_t {
        cudaError_t e;
        uint32_t* counters = reinterpret_cast<uint32_t*>(x.blob_dev + kBlobCounters);
        uint32_t* status = reinterpret_cast<uint32_t*>(x.blob_dev);
        if ((e = cudaMemsetAsync(counters, 0, 4 * kListGroups * kListCounters, c)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(x.fork, c)) != cudaSuccess) return e;
        const int nb = std::min<int>(kListBranches, static_cast<int>(keys.size()));
        for (int b = 0; b < nb; ++b)
            if ((e = cudaStreamWaitEvent(x.branch[b], x.fork, 0)) != cudaSuccess) return e;
        for (size_t g = 0; g < keys.size(); ++g) {
            cudaStream_t s = x.branch[g % kListBranches];
            const int D = keys[g] & 511, n_paths = (keys[g] >> 9) & 15;
            ListLaunch l{};
            l.status = status;
            l.D = D;
            l.s8 = ((keys[g] >> 13) & 1) != 0;
            l.ct62 = ((keys[g] >> 14) & 1) != 0;
            l.pair = n_paths >= 4;
            auto at = [&](int stage, int counter) {
                l.list = x.blob_dev + kBlobLists + (g * kListStages + stage) * kBlobListStride;
                l.next = counters + g * kListCounters + counter;
            };
            at(0, 0);
            l.grid = kCensusListPerSM * ctx->n_sm;
            if ((e = launch_census_list(l, s)) != cudaSuccess) return e;
            at(1, 1);
            l.grid = kCostListPerSM * ctx->n_sm;
            if ((e = launch_cost_list(l, s)) != cudaSuccess) return e;
            at(2, 2);
            l.grid = sweep_grid * ctx->n_sm;
            if ((e = launch_sweep_h_list(l, s)) != cudaSuccess) return e;
            const int vrx[3] = {1, -1, 0};
            const int nv = n_paths == 8 ? 3 : 1;
            for (int v = 0; v < nv; ++v) {
                at(3, 3 + v);
                l.rx = n_paths == 8 ? vrx[v] : 0;
                if ((e = launch_sweep_v_list(l, s)) != cudaSuccess) return e;
            }
            at(4, 6);
            l.grid = kMedianListPerSM * ctx->n_sm;
            if ((e = launch_median_list(l, s)) != cudaSuccess) return e;
        }
        for (int b = 0; b < nb; ++b) {
            if ((e = cudaEventRecord(x.join[b], x.branch[b])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(c, x.join[b], 0)) != cudaSuccess) return e;
        }
        return cudaMemcpyAsync(x.status_host, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, c);
    };
    const cudaError_t eb = body();
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c, &graph);
    if (eb != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(ctx, SGM_ECUDA, "capturing the batched graph: %s",
                    cudaGetErrorString(eb != cudaSuccess ? eb : ee));
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(ctx, SGM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    x.graphs.emplace(key, exec);
    *out = exec;
    return SGM_OK;
}

// The kernels a wave's graph launches.
static int wave_launches(const std::vector<BatchItem>& items, const std::vector<std::pair<size_t, size_t>>& groups) {
    int n = 0;
    for (const auto& g : groups) n += launches_per_group(items[g.first].p.n_paths);
    return n;
}

// The autotuner's key of a wave: its pairs' (W, H, D, n_paths), sorted.
static std::vector<int> wave_signature(const std::vector<BatchItem>& items, size_t b, size_t e) {
    std::vector<int> sig;
    for (size_t i = b; i < e; ++i) {
        sig.push_back(items[i].p.W);
        sig.push_back(items[i].p.H);
        sig.push_back(items[i].p.D | items[i].p.n_paths << 9);
    }
    std::vector<std::array<int, 3>> t(sig.size() / 3);
    for (size_t i = 0; i < t.size(); ++i) t[i] = {sig[3 * i], sig[3 * i + 1], sig[3 * i + 2]};
    std::sort(t.begin(), t.end());
    sig.clear();
    for (const auto& v : t) sig.insert(sig.end(), v.begin(), v.end());
    return sig;
}

// Enqueue the batched path for items[b, e) (one wave) on stream s: copy-in of
// host inputs, the lists, the wave's graph, copy-out of host outputs.
// `tune` (the caller's thread of sgm_compute_batch): on the first wave of its
// signature, time each sweep grid (one warm-up and kTuneReps runs, CUDA
// events on s) and keep the lowest median; without it (served batches) the
// default grid runs.
static int enqueue_wave(sgm_ctx* ctx, ListExec& x, std::vector<BatchItem>& items, size_t b, size_t e,
                        uint8_t* arena, cudaStream_t s, bool tune) {
    // the host image may be rewritten only once the previous wave's copy of it is done
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    for (size_t i = b; i < e; ++i) {
        BatchItem& it = items[i];
        const Layout l = layout_for(it.p, true);
        const size_t wh = static_cast<size_t>(it.p.W) * it.p.H;
        uint8_t* base = arena + it.offset;
        // host images go to the pair's arena region: pinned ones through a
        // staging kernel (each byte over the host link once), pageable ones
        // through cudaMemcpyAsync
        const uint8_t* st_src[2] = {nullptr, nullptr};
        uint8_t* st_dst[2] = {nullptr, nullptr};
        int n_st = 0;
        for (int side = 0; side < 2; ++side) {
            const uint8_t*& img = side ? it.right : it.left;
            if (is_device_ptr(img)) continue;
            uint8_t* dst = base + (side ? l.in_right : l.in_left);
            if (pointer_kind(img) == cudaMemoryTypeHost) {
                st_src[n_st] = img;
                st_dst[n_st++] = dst;
            } else {
                CUDA_TRY(ctx, cudaMemcpyAsync(dst, img, wh, cudaMemcpyHostToDevice, s));
            }
            img = dst;
        }
        if (n_st > 0) {
            CUDA_TRY(ctx, launch_stage(st_src[0], st_dst[0], st_src[1], st_dst[1], wh, s));
            ctx->launches += 1;
        }
    }
    const auto groups = wave_groups(items, b, e);
    std::vector<int> keys;
    for (const auto& g : groups) keys.push_back(group_code(items[g.first]));
    int rc = SGM_OK;
    const size_t used = build_lists(ctx, x, items, groups, arena, &rc);
    if (rc != SGM_OK) return rc;
    CUDA_TRY(ctx, cudaMemcpyAsync(x.blob_dev, x.blob_host, used, cudaMemcpyHostToDevice, s));
    const int per_wave = wave_launches(items, groups);
    int grid = kDefaultSweepGrid;  // served batches (the scheduler thread) take the default grid
    const std::vector<int> sig = tune ? wave_signature(items, b, e) : std::vector<int>{};
    if (tune && ctx->list_tuned.count(sig)) {
        grid = ctx->list_tuned[sig];
    } else if (tune) {
        float best = 0.0f;
        for (int cand : kSweepGrids) {
            cudaGraphExec_t g = nullptr;
            if ((rc = list_graph(ctx, x, keys, cand, &g)) != SGM_OK) return rc;
            std::vector<float> ms;
            for (int r = 0; r <= kTuneReps; ++r) {
                CUDA_TRY(ctx, cudaEventRecord(ctx->tune_ev[0], s));
                CUDA_TRY(ctx, cudaGraphLaunch(g, s));
                CUDA_TRY(ctx, cudaEventRecord(ctx->tune_ev[1], s));
                CUDA_TRY(ctx, cudaEventSynchronize(ctx->tune_ev[1]));
                ctx->launches += per_wave;
                float t = 0.0f;
                CUDA_TRY(ctx, cudaEventElapsedTime(&t, ctx->tune_ev[0], ctx->tune_ev[1]));
                if (r > 0) ms.push_back(t);  // run 0 warms up
            }
            std::sort(ms.begin(), ms.end());
            const float med = ms[ms.size() / 2];
            if (cand == kSweepGrids[0] || med < best) {
                best = med;
                grid = cand;
            }
        }
        ctx->list_tuned[sig] = grid;
    }
    cudaGraphExec_t g = nullptr;
    if ((rc = list_graph(ctx, x, keys, grid, &g)) != SGM_OK) return rc;
    CUDA_TRY(ctx, cudaGraphLaunch(g, s));
    ctx->launches += per_wave;
    for (size_t i = b; i < e; ++i) {
        const BatchItem& it = items[i];
        if (!is_device_ptr(it.out)) {
            const Layout l = layout_for(it.p, true);
            const size_t wh = static_cast<size_t>(it.p.W) * it.p.H;
            if (pointer_kind(it.out) == cudaMemoryTypeHost) {
                CUDA_TRY(ctx, launch_stage(arena + it.offset + l.out, it.out, nullptr, nullptr, wh, s));
                ctx->launches += 1;
            } else {
                CUDA_TRY(ctx, cudaMemcpyAsync(it.out, arena + it.offset + l.out, wh, cudaMemcpyDeviceToHost, s));
            }
        }
    }
    return SGM_OK;
}

// After a wave has finished: SGM_EDEVICE if a kernel rejected a descriptor.
static int wave_status(sgm_ctx* ctx, const ListExec& x) {
    const uint32_t st = *x.status_host;
    if (st != 0)
        return fail(ctx, SGM_EDEVICE, "a batched kernel rejected a work-list descriptor (device status %#x)", st);
    return SGM_OK;
}

// Run a batch through one arena: sort by group, pack waves that fit the
// budget (the context's memory cap, else the device's free memory plus what
// the arena already holds) and hold at most kListGroups groups, grow the arena
// once per wave.
static int run_batch(sgm_ctx* ctx, ListExec& x, std::vector<BatchItem>& items, uint8_t** arena, size_t* arena_bytes,
                     bool clear_graphs, cudaStream_t s, bool tune) {
    std::stable_sort(items.begin(), items.end(), [](const BatchItem& a, const BatchItem& c) {
        return batch_key(a) < batch_key(c);
    });
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(ctx, cudaMemGetInfo(&free_b, &total_b));
    size_t budget = (free_b + *arena_bytes) / 10 * 9;
    if (ctx->mem_cap) {
        const size_t other = ctx->serve_bytes.load();
        budget = std::min(budget, ctx->mem_cap > other ? ctx->mem_cap - other : 0);
    }
    size_t b = 0;
    while (b < items.size()) {
        size_t e = b, total = 0;
        int groups = 0;
        while (e < items.size()) {
            const size_t sz = layout_for(items[e].p, true).total;
            const bool new_group = e == b || batch_key(items[e]) != batch_key(items[e - 1]);
            if (e > b && (total + sz > budget || (new_group && groups == kListGroups))) break;
            groups += new_group ? 1 : 0;
            items[e].offset = total;
            total += sz;
            ++e;
        }
        if (total > budget)
            return fail(ctx, SGM_ENOMEM, "a %dx%d D=%d pair needs %zu bytes, over the memory budget of %zu", items[b].p.W,
                        items[b].p.H, items[b].p.D, total, budget);
        if (b > 0) {  // the previous wave still uses the arena
            CUDA_TRY(ctx, cudaStreamSynchronize(s));
            const int rc = wave_status(ctx, x);
            if (rc != SGM_OK) return rc;
        }
        int rc = ensure_arena(ctx, arena, arena_bytes, total, clear_graphs);
        if (rc != SGM_OK) return rc;
        rc = enqueue_wave(ctx, x, items, b, e, *arena, s, tune);
        if (rc != SGM_OK) return rc;
        b = e;
    }
    return SGM_OK;
}

// ---------------------------------------------------------------------------
// Served requests (continuous batching).  A scheduler thread owned by the
// context takes whatever is queued, in arrival order, as one batch for a free
// slot while the batch's buffers fit that slot's memory budget, and launches
// it through the batched path on the slot's stream; with kServeSlots slots,
// later arrivals are admitted and run while earlier batches are still on the
// GPU.  A stream callback marks a slot finished; the scheduler then retires
// its tickets and reuses the slot.
// ---------------------------------------------------------------------------
static void CUDART_CB slot_finished(void* data) {
    ServeSlot* sl = static_cast<ServeSlot*>(data);
    sgm_ctx* ctx = sl->ctx;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        sl->finished = true;
        sl->t_done = std::chrono::steady_clock::now();
    }
    ctx->cv_work.notify_all();
}

// Bytes a slot may hold for its next batch: the device's free memory plus the
// slot's own arena, at most a 1/kServeSlots share of the device, and within the
// context's memory cap after the other arenas.
static int slot_budget(sgm_ctx* ctx, const ServeSlot& sl, size_t* budget) {
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(ctx, cudaMemGetInfo(&free_b, &total_b));
    size_t b = std::min((free_b + sl.arena_bytes) / 10 * 9, total_b / 10 * 9 / kServeSlots);
    if (ctx->mem_cap) {
        const size_t other = ctx->arena_bytes + (ctx->serve_bytes.load() - sl.arena_bytes);
        b = std::min(b, ctx->mem_cap > other ? ctx->mem_cap - other : 0);
    }
    *budget = b;
    return SGM_OK;
}

static int slot_release(sgm_ctx* ctx, ServeSlot& sl) {
    if (!sl.arena) return SGM_OK;
    CUDA_TRY(ctx, cudaFreeAsync(sl.arena, sl.stream));
    ctx->serve_bytes -= sl.arena_bytes;
    sl.arena = nullptr;
    sl.arena_bytes = 0;
    return SGM_OK;
}

// Grow a slot's arena (stream-ordered, from the context's device pool),
// rounded up to a 64 MiB grain where the budget allows.
static int slot_reserve(sgm_ctx* ctx, ServeSlot& sl, size_t need, size_t budget) {
    if (sl.arena_bytes >= need) return SGM_OK;
    const size_t grain = size_t(64) << 20;
    need = std::max(need, std::min((need + grain - 1) / grain * grain, budget));
    int rc = slot_release(ctx, sl);
    if (rc != SGM_OK) return rc;
    void* p = nullptr;
    cudaError_t e = injected_alloc_failure(ctx) ? cudaErrorMemoryAllocation
                                                : cudaMallocFromPoolAsync(&p, need, ctx->serve_pool, sl.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SGM_ENOMEM, "served batch arena of %zu bytes: %s", need, cudaGetErrorString(e));
    }
    sl.arena = static_cast<uint8_t*>(p);
    sl.arena_bytes = need;
    ctx->serve_bytes += need;
    return SGM_OK;
}

// Enqueue one admitted batch on a slot; the callback fires after its copies.
static int slot_launch(sgm_ctx* ctx, ServeSlot& sl, size_t budget) {
    std::vector<BatchItem> items;
    items.reserve(sl.reqs.size());
    for (const Request& r : sl.reqs) items.push_back(BatchItem{r.p, r.left, r.right, r.out, 0});
    // pageable host buffers go through the slot's pinned staging
    auto pageable = [](const void* q) { return pointer_kind(q) == cudaMemoryTypeUnregistered; };
    size_t host = 0;
    for (const BatchItem& it : items) {
        const size_t wh = align_up(static_cast<size_t>(it.p.W) * it.p.H);
        host += (pageable(it.left) + pageable(it.right) + pageable(it.out)) * wh;
    }
    if (host > sl.pinned_bytes) {
        const size_t want = std::max(host, sl.pinned_bytes / 2 * 3);
        if (sl.pinned) CUDA_TRY(ctx, cudaFreeHost(sl.pinned));
        sl.pinned = nullptr;
        sl.pinned_bytes = 0;
        void* q = nullptr;
        CUDA_TRY(ctx, ctx_malloc_host(ctx, &q, want));
        sl.pinned = static_cast<uint8_t*>(q);
        sl.pinned_bytes = want;
    }
    sl.out_copies.clear();
    size_t off = 0;
    for (BatchItem& it : items) {
        const size_t wh = static_cast<size_t>(it.p.W) * it.p.H;
        if (pageable(it.left)) {
            std::memcpy(sl.pinned + off, it.left, wh);
            it.left = sl.pinned + off;
            off += align_up(wh);
        }
        if (pageable(it.right)) {
            std::memcpy(sl.pinned + off, it.right, wh);
            it.right = sl.pinned + off;
            off += align_up(wh);
        }
        if (pageable(it.out)) {
            sl.out_copies.emplace_back(it.out, sl.pinned + off, wh);
            it.out = sl.pinned + off;
            off += align_up(wh);
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const BatchItem& x, const BatchItem& y) {
        return batch_key(x) < batch_key(y);
    });
    size_t total = 0;
    for (BatchItem& it : items) {
        it.offset = total;
        total += layout_for(it.p, true).total;
    }
    int rc = slot_reserve(ctx, sl, total, budget);
    if (rc == SGM_OK) rc = enqueue_wave(ctx, sl.exec, items, 0, items.size(), sl.arena, sl.stream, false);
    if (rc == SGM_OK) CUDA_TRY(ctx, cudaLaunchHostFunc(sl.stream, slot_finished, &sl));
    return rc;
}

static double request_de(const Request& r) { return static_cast<double>(r.p.W) * r.p.H * r.p.D; }

static void retire(sgm_ctx* ctx, const std::vector<Request>& reqs, int rc,
                   std::chrono::steady_clock::time_point t_done) {
    for (const Request& r : reqs) {
        ctx->done[r.ticket] = rc;
        ctx->backlog_de = std::max(0.0, ctx->backlog_de - request_de(r));
        if (rc == SGM_OK) {
            ctx->latencies_us.push_back(std::chrono::duration<double, std::micro>(t_done - r.t_submit).count());
            ctx->served_de += request_de(r);
            ctx->lifetime_de += request_de(r);
        }
        --ctx->pending;
    }
}

// A batch leaves the GPU (under the context's lock): the busy time ends with the last one.
static void batch_left(sgm_ctx* ctx) {
    if (--ctx->in_flight == 0)
        ctx->busy_us +=
            std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - ctx->busy_since).count();
}

// Served disparity evaluations per microsecond of time with a batch in
// flight, or 0 before any batch has completed (under the context's lock).
static double service_rate(const sgm_ctx* ctx) {
    double busy = ctx->busy_us;
    if (ctx->in_flight > 0)
        busy += std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - ctx->busy_since).count();
    return (ctx->lifetime_de > 0.0 && busy > 0.0) ? ctx->lifetime_de / busy : 0.0;
}

// Estimated wait (us) of a request of `de` disparity evaluations submitted
// now, or -1 without a measured rate (under the context's lock).
static double estimated_wait_us(const sgm_ctx* ctx, double de) {
    const double rate = service_rate(ctx);
    return rate > 0.0 ? (ctx->backlog_de + de) / rate : -1.0;
}

static void serve_loop(sgm_ctx* ctx) {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto free_slot = [&]() -> ServeSlot* {  // the idle slot with the largest arena
        ServeSlot* best = nullptr;
        for (auto& sl : ctx->slots)
            if (!sl.busy && (!best || sl.arena_bytes > best->arena_bytes)) best = &sl;
        return best;
    };
    auto done_slot = [&]() -> ServeSlot* {
        for (auto& sl : ctx->slots)
            if (sl.busy && sl.finished) return &sl;
        return nullptr;
    };
    for (;;) {
        ctx->cv_work.wait(lk, [&] {
            return done_slot() || (ctx->stop && (!ctx->queue.empty() || ctx->in_flight == 0)) ||
                   (!ctx->stop && !ctx->queue.empty() && free_slot());
        });
        if (ServeSlot* sl = done_slot()) {
            lk.unlock();
            cudaError_t e = cudaStreamSynchronize(sl->stream);  // the callback has run: returns at once
            int rc = SGM_OK;
            if (e != cudaSuccess) rc = fail(ctx, SGM_ECUDA, "served batch: %s", cudaGetErrorString(e));
            if (rc == SGM_OK) rc = wave_status(ctx, sl->exec);
            if (rc == SGM_OK) rc = bounds_status(ctx);
            if (rc == SGM_OK)
                for (auto& c : sl->out_copies) std::memcpy(std::get<0>(c), std::get<1>(c), std::get<2>(c));
            lk.lock();
            retire(ctx, sl->reqs, rc, sl->t_done);
            sl->reqs.clear();
            sl->busy = sl->finished = false;
            batch_left(ctx);
            ctx->cv_done.notify_all();
            continue;
        }
        if (ctx->stop) {
            if (!ctx->queue.empty()) {
                const auto now = std::chrono::steady_clock::now();
                std::vector<Request> cancelled(ctx->queue.begin(), ctx->queue.end());
                ctx->queue.clear();
                retire(ctx, cancelled, SGM_ECANCELED, now);
                ctx->cv_done.notify_all();
            }
            if (ctx->in_flight == 0) return;
            continue;
        }
        // admission: reserve a slot, size its budget outside the lock, then take
        // queued requests in arrival order while they fit
        ServeSlot* sl = free_slot();
        sl->busy = true;
        lk.unlock();
        size_t budget = 0;
        int rc = slot_budget(ctx, *sl, &budget);
        lk.lock();
        size_t used = 0;
        std::set<std::tuple<int, int, bool, int>> keys;
        while (rc == SGM_OK && !ctx->queue.empty() && sl->reqs.size() < static_cast<size_t>(kServeMaxPairs)) {
            const Request& r = ctx->queue.front();
            const size_t sz = layout_for(r.p, true).total;
            const auto key = batch_key(BatchItem{r.p, nullptr, nullptr, nullptr, 0});
            if (used + sz > budget || (!keys.count(key) && keys.size() == static_cast<size_t>(kListGroups))) break;
            keys.insert(key);
            used += sz;
            sl->reqs.push_back(r);
            ctx->queue.pop_front();
        }
        if (rc == SGM_OK && sl->reqs.empty()) {
            if (ctx->in_flight > 0) {
                sl->busy = false;  // wait for a batch in flight to free memory
                ctx->cv_work.wait(lk, [&] { return done_slot() != nullptr || ctx->stop; });
                continue;
            }
            // nothing runs: give the memory of the other idle arenas back and retry
            bool released = false;
            for (auto& o : ctx->slots) {
                if (&o != sl && o.arena) {
                    lk.unlock();
                    slot_release(ctx, o);
                    cudaStreamSynchronize(o.stream);
                    lk.lock();
                    released = true;
                }
            }
            if (released) {
                sl->busy = false;
                continue;
            }
            // nothing runs and the oldest request alone exceeds the budget
            std::vector<Request> one{ctx->queue.front()};
            ctx->queue.pop_front();
            rc = fail(ctx, SGM_ENOMEM, "served %dx%d D=%d pair exceeds the memory budget of %zu bytes", one[0].p.W,
                      one[0].p.H, one[0].p.D, budget);
            retire(ctx, one, rc, std::chrono::steady_clock::now());
            sl->busy = false;
            ctx->cv_done.notify_all();
            continue;
        }
        if (rc != SGM_OK) {  // the budget query failed: fail what is queued
            std::vector<Request> failed(ctx->queue.begin(), ctx->queue.end());
            ctx->queue.clear();
            retire(ctx, failed, rc, std::chrono::steady_clock::now());
            sl->busy = false;
            ctx->cv_done.notify_all();
            continue;
        }
        if (ctx->in_flight++ == 0) ctx->busy_since = std::chrono::steady_clock::now();
        ctx->max_in_flight = std::max(ctx->max_in_flight, ctx->in_flight);
        ++ctx->batches;
        ctx->batched_pairs += sl->reqs.size();
        lk.unlock();
        rc = slot_launch(ctx, *sl, budget);
        lk.lock();
        if (rc != SGM_OK) {
            cudaStreamSynchronize(sl->stream);
            retire(ctx, sl->reqs, rc, std::chrono::steady_clock::now());
            sl->reqs.clear();
            sl->busy = sl->finished = false;
            batch_left(ctx);
            ctx->cv_done.notify_all();
        }
    }
}

extern "C" {

int sgm_create(sgm_ctx** out, int device, size_t mem_cap_bytes, unsigned flags) {
    if (!out) return fail(nullptr, SGM_EINVAL, "null output pointer");
    *out = nullptr;
    if (flags & ~(SGM_FLAG_STAGE_TIMING | SGM_FLAG_CENSUS_FULL))
        return fail(nullptr, SGM_EINVAL, "unknown flags %#x", flags);
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return fail(nullptr, SGM_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= n) return fail(nullptr, SGM_EINVAL, "device %d out of range [0, %d)", device, n);
    if ((e = cudaSetDevice(device)) != cudaSuccess)
        return fail(nullptr, SGM_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    sgm_ctx* ctx = new sgm_ctx();
    ctx->device = device;
    ctx->mem_cap = mem_cap_bytes;
    if ((e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming)) != cudaSuccess) {
        sgm_destroy(ctx);
        return fail(nullptr, SGM_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    for (auto& sl : ctx->slots) {
        sl.ctx = ctx;
        if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess) {
            sgm_destroy(ctx);
            return fail(nullptr, SGM_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
    }
    {
        // the served arenas come from a pool that keeps freed memory resident
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        uint64_t keep = UINT64_MAX;
        if ((e = cudaMemPoolCreate(&ctx->serve_pool, &props)) != cudaSuccess ||
            (e = cudaMemPoolSetAttribute(ctx->serve_pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            sgm_destroy(ctx);
            return fail(nullptr, SGM_ECUDA, "device memory pool: %s", cudaGetErrorString(e));
        }
    }
    if ((e = init_kernel_attributes()) != cudaSuccess) {
        sgm_destroy(ctx);
        return fail(nullptr, SGM_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
    }
    if ((e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) {
        sgm_destroy(ctx);
        return fail(nullptr, SGM_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    }
    if (const char* v = std::getenv("SGM_TEST_FAIL_ALLOC")) ctx->fail_alloc_at = std::atoi(v);
    if (const char* v = std::getenv("SGM_TEST_BAD_JOB")) ctx->bad_job_waves = std::atoi(v);
#ifdef SGM_BOUNDS_CHECK
    if (const char* v = std::getenv("SGM_TEST_BOUNDS_SHRINK")) ctx->bounds_shrink = std::atoi(v) != 0;
#endif
    {
        int rc = list_exec_init(ctx, ctx->batch_exec);
        for (auto& sl : ctx->slots)
            if (rc == SGM_OK) rc = list_exec_init(ctx, sl.exec);
        if (rc != SGM_OK) {
            const std::string why = ctx->err;
            sgm_destroy(ctx);
            return fail(nullptr, rc, "%s", why.c_str());
        }
    }
    ctx->stream = ctx->own_stream;
    ctx->stage_timing = (flags & SGM_FLAG_STAGE_TIMING) != 0;
    ctx->ct62 = (flags & SGM_FLAG_CENSUS_FULL) ? 1 : 0;
    if (ctx->stage_timing) {
        for (auto& ev : ctx->stage_ev) {
            if ((e = cudaEventCreate(&ev)) != cudaSuccess) {
                sgm_destroy(ctx);
                return fail(nullptr, SGM_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
            }
        }
    }
    for (auto& ev : ctx->tune_ev) {
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) {
            sgm_destroy(ctx);
            return fail(nullptr, SGM_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
        }
    }
    *out = ctx;
    return SGM_OK;
}

int sgm_destroy(sgm_ctx* ctx) {
    if (!ctx) return SGM_OK;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->stop = true;
    }
    ctx->cv_work.notify_all();
    if (ctx->worker.joinable()) ctx->worker.join();
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    if (ctx->arena) cudaFree(ctx->arena);
    list_exec_release(ctx->batch_exec);
    for (auto& sl : ctx->slots) {
        if (sl.arena) cudaFreeAsync(sl.arena, sl.stream);
        if (sl.pinned) cudaFreeHost(sl.pinned);
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            cudaStreamDestroy(sl.stream);
        }
        list_exec_release(sl.exec);
    }
    if (ctx->serve_pool) cudaMemPoolDestroy(ctx->serve_pool);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->aux_stream) {
        cudaStreamSynchronize(ctx->aux_stream);
        cudaStreamDestroy(ctx->aux_stream);
    }
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    for (auto& ev : ctx->stage_ev)
        if (ev) cudaEventDestroy(ev);
    for (auto& ev : ctx->tune_ev)
        if (ev) cudaEventDestroy(ev);
    delete ctx;
    return SGM_OK;
}

const char* sgm_last_error(const sgm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_noctx_err.c_str(); }

int sgm_set_stream(sgm_ctx* ctx, void* cuda_stream) {
    if (!ctx) return fail(nullptr, SGM_EINVAL, "null context");
    ctx->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->own_stream;
    return SGM_OK;
}

int sgm_compute(sgm_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H, int D, int P1, int P2,
                int n_paths, uint8_t* disp_out) {
    const Problem p = make_problem(ctx, W, H, D, P1, P2, n_paths);
    int rc = check_args(ctx, p, left, right, disp_out);
    if (rc != SGM_OK) return rc;
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    rc = ensure_arena(ctx, &ctx->arena, &ctx->arena_bytes, arena_need(p), true);
    if (rc != SGM_OK) return rc;
    rc = enqueue_pair(ctx, p, ctx->arena, left, right, disp_out, ctx->stream, true);
    if (rc != SGM_OK) return rc;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return bounds_status(ctx);
}

int sgm_compute_ex(sgm_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H, int D, int P1, int P2,
                   int n_paths, unsigned post, uint16_t* disp16_out) {
    Problem p = make_problem(ctx, W, H, D, P1, P2, n_paths);
    p.post = (post & ~static_cast<unsigned>(kPostOut16)) == post ? static_cast<int>(post) | kPostOut16 : -1;
    int rc = check_args(ctx, p, left, right, disp16_out);
    if (rc != SGM_OK) return rc;
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    rc = ensure_arena(ctx, &ctx->arena, &ctx->arena_bytes, layout_for(p).total, true);
    if (rc != SGM_OK) return rc;
    rc = enqueue_pair(ctx, p, ctx->arena, left, right, reinterpret_cast<uint8_t*>(disp16_out), ctx->stream, true);
    if (rc != SGM_OK) return rc;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return bounds_status(ctx);
}

int sgm_compute_async(sgm_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H, int D, int P1, int P2,
                      int n_paths, uint8_t* disp_out) {
    const Problem p = make_problem(ctx, W, H, D, P1, P2, n_paths);
    int rc = check_args(ctx, p, left, right, disp_out);
    if (rc != SGM_OK) return rc;
    if (!is_device_ptr(left) || !is_device_ptr(right) || !is_device_ptr(disp_out))
        return fail(ctx, SGM_EINVAL, "sgm_compute_async takes device pointers only");
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    rc = ensure_arena(ctx, &ctx->arena, &ctx->arena_bytes, arena_need(p), true);
    if (rc != SGM_OK) return rc;
    Problem q = p;
    rc = choose_schedule(ctx, q, ctx->arena, left, right, disp_out, ctx->stream);
    if (rc != SGM_OK) return rc;
    return enqueue_graph(ctx, q, ctx->arena, left, right, disp_out, ctx->stream);
}

int sgm_compute_ex_async(sgm_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H, int D, int P1,
                         int P2, int n_paths, unsigned post, uint16_t* disp16_out) {
    Problem p = make_problem(ctx, W, H, D, P1, P2, n_paths);
    p.post = (post & ~static_cast<unsigned>(kPostOut16)) == post ? static_cast<int>(post) | kPostOut16 : -1;
    int rc = check_args(ctx, p, left, right, disp16_out);
    if (rc != SGM_OK) return rc;
    if (!is_device_ptr(left) || !is_device_ptr(right) || !is_device_ptr(disp16_out))
        return fail(ctx, SGM_EINVAL, "sgm_compute_ex_async takes device pointers only");
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    rc = ensure_arena(ctx, &ctx->arena, &ctx->arena_bytes, layout_for(p).total, true);
    if (rc != SGM_OK) return rc;
    return enqueue_graph(ctx, p, ctx->arena, left, right, reinterpret_cast<uint8_t*>(disp16_out), ctx->stream);
}

int sgm_compute_batch(sgm_ctx* ctx, int n, const sgm_pair* pairs) {
    if (!ctx) return fail(nullptr, SGM_EINVAL, "null context");
    if (n < 0 || (n > 0 && !pairs)) return fail(ctx, SGM_EINVAL, "bad batch (n=%d, pairs=%p)", n, (const void*)pairs);
    std::vector<BatchItem> items;
    items.reserve(n);
    for (int i = 0; i < n; ++i) {
        const sgm_pair& q = pairs[i];
        const Problem p = make_problem(ctx, q.W, q.H, q.D, q.P1, q.P2, q.n_paths);
        int rc = check_args(ctx, p, q.left, q.right, q.disp_out);
        if (rc != SGM_OK) return fail(ctx, rc, "pair %d: %s", i, ctx->err.c_str());
        items.push_back(BatchItem{p, q.left, q.right, q.disp_out, 0});
    }
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int rc = run_batch(ctx, ctx->batch_exec, items, &ctx->arena, &ctx->arena_bytes, true, ctx->stream, true);
    if (rc != SGM_OK) return rc;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    rc = wave_status(ctx, ctx->batch_exec);
    return rc != SGM_OK ? rc : bounds_status(ctx);
}

int sgm_submit(sgm_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H, int D, int P1, int P2,
               int n_paths, uint8_t* disp_out, uint64_t* ticket) {
    const Problem p = make_problem(ctx, W, H, D, P1, P2, n_paths);
    int rc = check_args(ctx, p, left, right, disp_out);
    if (rc != SGM_OK) return rc;
    if (!ticket) return fail(ctx, SGM_EINVAL, "null ticket pointer");
    if (ctx->mem_cap && layout_for(p, true).total + ctx->arena_bytes > ctx->mem_cap)
        return fail(ctx, SGM_ENOMEM, "pair %dx%d D=%d needs more than the context's memory cap", W, H, D);
    std::lock_guard<std::mutex> lk(ctx->mu);
    const double de = static_cast<double>(W) * H * D;
    if (ctx->admit_max_us > 0) {
        const double wait = estimated_wait_us(ctx, de);
        if (wait > static_cast<double>(ctx->admit_max_us)) {
            ++ctx->shed;
            return fail(ctx, SGM_EAGAIN, "estimated wait %.0f us exceeds the admission bound of %lld us", wait,
                        static_cast<long long>(ctx->admit_max_us));
        }
    }
    if (!ctx->worker_started) {
        ctx->worker = std::thread(serve_loop, ctx);
        ctx->worker_started = true;
    }
    Request r{ctx->next_ticket++, p, left, right, disp_out, std::chrono::steady_clock::now()};
    *ticket = r.ticket;
    ctx->backlog_de += de;
    ctx->queue.push_back(r);
    ctx->outstanding.insert(r.ticket);
    ++ctx->pending;
    ctx->cv_work.notify_one();
    return SGM_OK;
}

int sgm_poll(sgm_ctx* ctx, uint64_t ticket, int64_t timeout_us) {
    if (!ctx) return fail(nullptr, SGM_EINVAL, "null context");
    std::unique_lock<std::mutex> lk(ctx->mu);
    if (!ctx->outstanding.count(ticket))
        return fail(ctx, SGM_EINVAL, "unknown or already retired ticket %llu", (unsigned long long)ticket);
    auto ready = [&] { return ctx->done.count(ticket) != 0; };
    if (!ready()) {
        if (timeout_us == 0) return SGM_EAGAIN;
        if (timeout_us < 0) {
            ctx->cv_done.wait(lk, ready);
        } else if (!ctx->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
            return SGM_ETIMEDOUT;
        }
    }
    const int rc = ctx->done[ticket];
    ctx->done.erase(ticket);
    ctx->outstanding.erase(ticket);
    return rc;
}

int sgm_served_stats(sgm_ctx* ctx, double* out, int n_out) {
    if (!ctx || !out || n_out < 4) return fail(ctx, SGM_EINVAL, "sgm_served_stats needs a context and 4 outputs");
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::vector<double> v = ctx->latencies_us;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, static_cast<size_t>(f * v.size()))]; };
    out[0] = static_cast<double>(v.size());
    out[1] = q(0.50);
    out[2] = q(0.99);
    out[3] = v.empty() ? 0.0 : v.back();
    if (n_out >= 8) {
        out[4] = static_cast<double>(ctx->batches);
        out[5] = ctx->batches ? static_cast<double>(ctx->batched_pairs) / ctx->batches : 0.0;
        out[6] = static_cast<double>(ctx->max_in_flight);
        out[7] = ctx->served_de;
    }
    if (n_out >= 10) {
        out[8] = static_cast<double>(ctx->shed);
        out[9] = service_rate(ctx) * 1e6;
    }
    if (n_out >= 13) {
        out[10] = static_cast<double>(ctx->queue.size());  // queued, not yet admitted
        out[11] = static_cast<double>(ctx->in_flight);
        out[12] = static_cast<double>(ctx->serve_bytes.load());  // device bytes of the slots' arenas
    }
    return SGM_OK;
}

// The tuning cache: {"sgm_tuning": 1, "sm_count": N, "schedules": [[W, H, D,
// n_paths, ct62, s8, schedule], ...], "batch_grids": [[grid, W, H, D | paths
// << 9, ...], ...]}.  The reader takes the integers of each bracketed list in
// order.
int sgm_save_tuning(const sgm_ctx* ctx, const char* path) {
    if (!ctx || !path) return fail(nullptr, SGM_EINVAL, "null context or path");
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(const_cast<sgm_ctx*>(ctx), SGM_EINVAL, "cannot write %s", path);
    std::fprintf(f, "{\"sgm_tuning\": 1, \"sm_count\": %d, \"schedules\": [", ctx->n_sm);
    bool first = true;
    for (const auto& kv : ctx->tuned) {
        const auto& k = kv.first;
        std::fprintf(f, "%s[%d, %d, %d, %d, %d, %d, %d]", first ? "" : ", ", std::get<0>(k), std::get<1>(k),
                     std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k) ? 1 : 0, kv.second);
        first = false;
    }
    std::fprintf(f, "], \"batch_grids\": [");
    first = true;
    for (const auto& kv : ctx->list_tuned) {
        std::fprintf(f, "%s[%d", first ? "" : ", ", kv.second);
        for (int v : kv.first) std::fprintf(f, ", %d", v);
        std::fprintf(f, "]");
        first = false;
    }
    std::fprintf(f, "]}\n");
    const bool ok = std::fclose(f) == 0;
    return ok ? SGM_OK : fail(const_cast<sgm_ctx*>(ctx), SGM_EINVAL, "cannot write %s", path);
}

// The integer lists inside the outer list that follows `"key":` in text.
static bool read_lists(const std::string& text, const char* key, std::vector<std::vector<long>>* out) {
    const std::string k = std::string("\"") + key + "\"";
    size_t i = text.find(k);
    if (i == std::string::npos) return false;
    i = text.find('[', i + k.size());
    if (i == std::string::npos) return false;
    int depth = 0;
    std::vector<long> cur;
    for (size_t j = i; j < text.size(); ++j) {
        const char c = text[j];
        if (c == '[') {
            ++depth;
            if (depth == 2) cur.clear();
            if (depth > 2) return false;
        } else if (c == ']') {
            if (depth == 2) out->push_back(cur);
            if (--depth == 0) return true;
        } else if (depth == 2 && (c == '-' || (c >= '0' && c <= '9'))) {
            char* end = nullptr;
            cur.push_back(std::strtol(text.c_str() + j, &end, 10));
            j = static_cast<size_t>(end - text.c_str()) - 1;
        } else if (!(c == ',' || c == ' ' || c == '\n' || c == '\t' || c == '\r')) {
            return false;
        }
    }
    return false;
}

int sgm_load_tuning(sgm_ctx* ctx, const char* path) {
    if (!ctx || !path) return fail(ctx, SGM_EINVAL, "null context or path");
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(ctx, SGM_EINVAL, "cannot read %s", path);
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
    std::fclose(f);
    const size_t h = text.find("\"sm_count\":");
    if (text.find("\"sgm_tuning\": 1") == std::string::npos || h == std::string::npos)
        return fail(ctx, SGM_EINVAL, "%s is not a tuning cache", path);
    if (std::atoi(text.c_str() + h + 11) != ctx->n_sm)
        return fail(ctx, SGM_EINVAL, "%s was tuned on a device with another SM count", path);
    std::vector<std::vector<long>> sched, grids;
    if (!read_lists(text, "schedules", &sched) || !read_lists(text, "batch_grids", &grids))
        return fail(ctx, SGM_EINVAL, "%s is malformed", path);
    for (const auto& v : sched) {
        if (v.size() != 7 || v[6] < 0 || v[6] > SGM_SCHED_PAIRS)
            return fail(ctx, SGM_EINVAL, "%s: bad schedule entry", path);
    }
    for (const auto& v : grids) {
        bool known = false;
        for (int g : kSweepGrids) known |= v.size() >= 4 && v[0] == g;
        if (!known || (v.size() - 1) % 3 != 0) return fail(ctx, SGM_EINVAL, "%s: bad batch grid entry", path);
    }
    for (const auto& v : sched)
        ctx->tuned[std::make_tuple(int(v[0]), int(v[1]), int(v[2]), int(v[3]), int(v[4]), v[5] != 0)] = int(v[6]);
    for (const auto& v : grids) ctx->list_tuned[std::vector<int>(v.begin() + 1, v.end())] = int(v[0]);
    return SGM_OK;
}

int sgm_set_admission_bound(sgm_ctx* ctx, int64_t max_wait_us) {
    if (!ctx) return fail(nullptr, SGM_EINVAL, "null context");
    if (max_wait_us < 0) return fail(ctx, SGM_EINVAL, "negative admission bound %lld", (long long)max_wait_us);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->admit_max_us = max_wait_us;
    return SGM_OK;
}

int sgm_served_reset_stats(sgm_ctx* ctx) {
    if (!ctx) return fail(nullptr, SGM_EINVAL, "null context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->latencies_us.clear();
    ctx->batches = ctx->batched_pairs = 0;
    ctx->shed = 0;
    ctx->max_in_flight = ctx->in_flight;
    ctx->served_de = 0.0;
    return SGM_OK;
}

int sgm_debug_stages(sgm_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H, int D, int P1, int P2,
                     int n_paths, void* Fb, void* Fm, uint8_t* MC, uint16_t* S, uint8_t* raw, uint8_t* disp) {
    Problem p = make_problem(ctx, W, H, D, P1, P2, n_paths);
    if (ctx && n_paths == 4 && ctx->forced_sched >= 0) p.sched = ctx->forced_sched;  // else the first schedule
    int rc = check_args(ctx, p, left, right, left);
    if (rc != SGM_OK) return rc;
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (pairs_sched(p) && !pairs_fit(p)) return fail(ctx, SGM_EINVAL, "problem too large for the paired schedule");
    const Layout l = layout_for(p);
    const size_t wh = static_cast<size_t>(W) * H;
    const size_t extra = align_up(wh * D * 2) + align_up(wh * D) + align_up(wh);
    rc = ensure_arena(ctx, &ctx->arena, &ctx->arena_bytes, l.total + extra, true);
    if (rc != SGM_OK) return rc;
    uint8_t* a = ctx->arena;
    uint16_t* Sdev = reinterpret_cast<uint16_t*>(a + l.total);
    uint8_t* MCnat = a + l.total + align_up(wh * D * 2);
    uint8_t* rawnat = MCnat + align_up(wh * D);
    cudaStream_t s = ctx->stream;
    CUDA_TRY(ctx, cudaMemcpyAsync(a + l.in_left, left, wh, cudaMemcpyHostToDevice, s));
    CUDA_TRY(ctx, cudaMemcpyAsync(a + l.in_right, right, wh, cudaMemcpyHostToDevice, s));
    CUDA_TRY(ctx, enqueue_path(ctx, p, a, a + l.in_left, a + l.in_right, a + l.out, S ? Sdev : nullptr, s, false));
    const size_t fbytes = (p.ct62 ? 8 : 4) * wh;
    if (Fb) CUDA_TRY(ctx, cudaMemcpyAsync(Fb, a + l.Fb, fbytes, cudaMemcpyDeviceToHost, s));
    if (Fm) CUDA_TRY(ctx, cudaMemcpyAsync(Fm, a + l.Fm, fbytes, cudaMemcpyDeviceToHost, s));
    if (MC) {
        if (pairs_sched(p))
            CUDA_TRY(ctx, launch_unquad_cost(a + l.rec, l.RB, MCnat, W, H, D, s));
        else
            CUDA_TRY(ctx, launch_unpair_cost(a + l.rec, l.RB, MCnat, W, H, D, s));
        CUDA_TRY(ctx, cudaMemcpyAsync(MC, MCnat, wh * D, cudaMemcpyDeviceToHost, s));
    }
    if (S) CUDA_TRY(ctx, cudaMemcpyAsync(S, Sdev, 2 * wh * D, cudaMemcpyDeviceToHost, s));
    if (raw && pairs_sched(p)) {
        // quads of bytes: the cost unquad with one "disparity" per pixel
        CUDA_TRY(ctx, launch_unquad_cost(a + l.raw, 4, rawnat, W, H, 1, s));
        CUDA_TRY(ctx, cudaMemcpyAsync(raw, rawnat, wh, cudaMemcpyDeviceToHost, s));
    } else if (raw) {
        CUDA_TRY(ctx, cudaMemcpyAsync(raw, a + l.raw, wh, cudaMemcpyDeviceToHost, s));
    }
    if (disp) CUDA_TRY(ctx, cudaMemcpyAsync(disp, a + l.out, wh, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return bounds_status(ctx);
}

int sgm_stage_times(sgm_ctx* ctx, float* ms_out, int n) {
    if (!ctx) return fail(nullptr, SGM_EINVAL, "null context");
    if (!ctx->stage_timing) return fail(ctx, SGM_EINVAL, "context was created without SGM_FLAG_STAGE_TIMING");
    const int k = ctx->last_stages;
    if (k == 0) return fail(ctx, SGM_EINVAL, "no path has been enqueued yet");
    CUDA_TRY(ctx, cudaEventSynchronize(ctx->stage_ev[k]));
    for (int i = 0; i < k && i < n; ++i) CUDA_TRY(ctx, cudaEventElapsedTime(&ms_out[i], ctx->stage_ev[i], ctx->stage_ev[i + 1]));
    return k;
}

int sgm_stage_paths(const sgm_ctx* ctx) { return ctx ? ctx->last_n_paths : 0; }

const char* sgm_stage_label(const sgm_ctx* ctx, int i) {
    if (!ctx || ctx->last_n_paths == 0) return nullptr;
    if (ctx->last_n_paths == 4 && ctx->last_sched == SGM_SCHED_H_THEN_V) {
        static const char* four_hv[] = {"census", "cost", "sweep_h+v1", "sweep_v2", "median"};
        return (i >= 0 && i < 5) ? four_hv[i] : nullptr;
    }
    if (ctx->last_n_paths == 4 && ctx->last_sched == SGM_SCHED_PAIRS) {
        static const char* four_pairs[] = {"census", "cost", "pairs_vh", "pairs_h_wta", "median"};
        return (i >= 0 && i < 5) ? four_pairs[i] : nullptr;
    }
    return sgm_stage_name(ctx->last_n_paths, i);
}

int sgm_set_schedule(sgm_ctx* ctx, int schedule) {
    if (!ctx) return fail(nullptr, SGM_EINVAL, "null context");
    if (schedule < -1 || schedule > SGM_SCHED_PAIRS) return fail(ctx, SGM_EINVAL, "unknown schedule %d", schedule);
    ctx->forced_sched = schedule;
    return SGM_OK;
}

int sgm_schedule_for(const sgm_ctx* ctx, int W, int H, int D, int P1, int P2, int n_paths) {
    if (!ctx) return SGM_EINVAL;
    if (n_paths != 4) return SGM_SCHED_V_THEN_H;
    if (ctx->forced_sched >= 0) return ctx->forced_sched;
    Problem p = make_problem(ctx, W, H, D, P1, P2, n_paths);
    auto it = ctx->tuned.find(std::make_tuple(p.W, p.H, p.D, p.n_paths, p.ct62, s8_for(p)));
    return it == ctx->tuned.end() ? -1 : it->second;
}

const char* sgm_stage_name(int n_paths, int i) {
    // 2 paths: "sweep_h" (left to right), "sweep_v" (top to bottom with Eq. 4).
    // 4 paths: "sweep_v+h1" (the whole vertical pair beside the horizontal
    // first halves), "sweep_h2" (the horizontal second halves with Eq. 4).
    // 8 paths: "sweep_h" (the horizontal pair with the first halves of the
    // three vertical-type pairs), then one launch per second half.
    static const char* two[] = {"census", "cost", "sweep_h", "sweep_v", "median"};
    static const char* four[] = {"census", "cost", "sweep_v+h1", "sweep_h2", "median"};
    static const char* eight[] = {"census", "cost", "sweep_h", "sweep_diag+", "sweep_diag-", "sweep_v", "median"};
    if (n_paths == 8) return (i >= 0 && i < 7) ? eight[i] : nullptr;
    if (n_paths == 4) return (i >= 0 && i < 5) ? four[i] : nullptr;
    if (n_paths == 2) return (i >= 0 && i < 5) ? two[i] : nullptr;
    return nullptr;
}

uint64_t sgm_kernel_launches(const sgm_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

int sgm_bounds_checked(void) {
#ifdef SGM_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

unsigned sgm_bounds_fault(void) { return take_bounds_fault(); }

const char* sgm_version(void) { return "sgm-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point (sgm_compute_static).
//
// Every intermediate of the path lives in one file-scope device array of
// kStaticScratchBytes, which each GPU that loads this library keeps until the
// process exits.  Host code may not use `g_static_scratch` as an address (it
// is a host-side stand-in); the device address is looked up once per device
// with cudaGetSymbolAddress while that device is current.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = size_t(48) << 20;  // 48 MiB
__device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
uint8_t* g_static_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device (set-up on the
// first call per device).
cudaError_t static_scratch_for_current_device(uint8_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return e;
        e = init_kernel_attributes();
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = static_cast<uint8_t*>(ptr);
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

// What the allocation-free path touches: features, records with one stored-L_r
// field (every pair runs both phases in one launch) and the raw disparity.
Layout static_layout(const Problem& p) {
    const size_t wh = static_cast<size_t>(p.W) * p.H;
    Layout l{};
    l.n_lx = p.n_paths == 2 ? 0 : 1;
    l.RB = record_bytes(p.D, false, l.n_lx);
    size_t o = 0;
    l.Fb = o;
    o = align_up(o + 4 * wh);
    l.Fm = o;
    o = align_up(o + 4 * wh);
    l.rec = o;
    o = align_up(o + wh * static_cast<size_t>(l.RB));
    l.raw = o;
    o = align_up(o + wh);
    l.total = o;
    return l;
}

// The path of Section 2, stages 2-4, with every phase on one stream.
cudaError_t enqueue_path_static(const Problem& p, uint8_t* arena, const uint8_t* left, const uint8_t* right,
                                uint8_t* disp, cudaStream_t s) {
    const Layout l = static_layout(p);
    void* Fb = arena + l.Fb;
    void* Fm = arena + l.Fm;
    cudaError_t e;
    if ((e = launch_census(left, right, Fb, Fm, p.W, p.H, false, s)) != cudaSuccess) return e;
    if ((e = launch_cost(Fb, Fm, arena + l.rec, l.RB, p.W, p.H, p.D, false, s)) != cudaSuccess) return e;
    SweepArgs a{};
    a.rec = arena + l.rec;
    a.RB = l.RB;
    a.lx_off = 3 * p.D;  // every pair runs both phases in one launch: field 0 serves them in turn
    a.raw = arena + l.raw;
    a.W = p.W;
    a.H = p.H;
    a.D = p.D;
    a.P1x2 = static_cast<uint32_t>(p.P1) * 0x10001u;
    a.P2x2 = static_cast<uint32_t>(p.P2) * 0x10001u;
    a.pair = p.n_paths >= 4;
    a.s8 = s8_for(p);
    if ((e = launch_sweep_h(a, s)) != cudaSuccess) return e;
    if (!a.pair) {
        a.wta = 1;
        if ((e = launch_sweep_v(a, s)) != cudaSuccess) return e;
    } else {
        const int vrx[3] = {1, -1, 0};
        const int* rxs = p.n_paths == 8 ? vrx : vrx + 2;
        const int nv = p.n_paths == 8 ? 3 : 1;
        for (int v = 0; v < nv; ++v) {  // both phases of each vertical-type pair in one launch
            SweepArgs b = a;
            b.rx = rxs[v];
            b.wta = (rxs[v] == 0) ? 1 : 0;
            b.phase = 0;
            if ((e = launch_sweep_v(b, s)) != cudaSuccess) return e;
        }
    }
    return launch_median(a.raw, disp, p.W, p.H, s);
}

}  // namespace

extern "C" int sgm_compute_static(const uint8_t* left, const uint8_t* right, int W, int H, int D, int P1, int P2,
                                  int n_paths, uint8_t* disp_out, void* cuda_stream) {
    const Problem p{W, H, D, P1, P2, n_paths};  // CSCT features
    if (!left || !right || !disp_out) return fail(nullptr, SGM_EINVAL, "null image or output pointer");
    std::string why;
    if (!valid_problem(p, &why)) return fail(nullptr, SGM_EINVAL, "%s", why.c_str());
    if (!is_device_ptr(left) || !is_device_ptr(right) || !is_device_ptr(disp_out))
        return fail(nullptr, SGM_EINVAL, "sgm_compute_static takes device pointers only");
    const size_t need = static_layout(p).total;
    if (need > kStaticScratchBytes)
        return fail(nullptr, SGM_EINVAL,
                    "%dx%d D=%d with %d paths needs %zu bytes of scratch; the static scratch holds %zu bytes", W, H, D,
                    n_paths, need, kStaticScratchBytes);
    uint8_t* scratch = nullptr;
    cudaError_t e = static_scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return fail(nullptr, SGM_ECUDA, "static scratch set-up: %s", cudaGetErrorString(e));
    e = enqueue_path_static(p, scratch, left, right, disp_out, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return fail(nullptr, SGM_ECUDA, "sgm_compute_static: %s", cudaGetErrorString(e));
    return SGM_OK;
}
