// Host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sgm {

// The sweeps keep every per-(pixel, disparity) cube of a pair in one array of
// per-pixel records [H][W][RB] bytes: the paired costs MC (D bytes, offset 0),
// the sums S (offset D: D paired bytes when s8, else D/2 packed u16x2 words),
// then one stored-L_r field (D paired bytes) per pair of opposite paths that
// needs its own.  One offset then addresses every field of a step's pixel.
inline int record_bytes(int D, bool s8, int n_lx) { return D + (s8 ? D : 2 * D) + n_lx * D; }

// Arguments of the aggregation sweeps (Eq. 3) over one pair.
struct SweepArgs {
    uint8_t* rec;       // per-pixel records [H][W][RB]
    uint8_t* raw;       // winner-take-all disparity [H][W] (final vertical sweep)
    uint16_t* Sdbg;     // optional natural-order S [H][W][D] (debug)
    int RB;             // record bytes (W * H * RB < 2^32)
    int lx_off;         // byte offset of this pair's stored-L_r field in a record
    int W, H, D;
    uint32_t P1x2, P2x2;  // penalties replicated in both u16 halves
    int rx;               // vertical-type sweeps: 0 (vertical), +1 / -1 (diagonals)
    int pair;             // 1: both opposite directions, 0: the forward one only
    int wta;              // vertical-type sweeps: 1 = finish with Eq. 4, 0 = add into S
    int phase;            // vertical-type pairs: 0 = both phases, 1 = first half of each path
                          // (saves the path state), 2 = second half (restores it)
    uint32_t* state;      // path states between phases 1 and 2 (sweep_state_words)
    uint32_t* state_end;  // the end of the state array (bounds-checked build)
    int s8;               // S kept as paired bytes instead of u16x2 words
    // Post-filter form of the sweeps (sgm_compute_ex): post = 1 selects it.
    // Every step q -> p then takes its jump penalty from a per-block table
    // indexed by |I(p) - I(q)| of the base image img (max(P1, P2 / (1 + g))
    // with ap2, else P2 throughout), and a winner-take-all sweep with
    // sub != nullptr also writes, per pixel, S(d-1) - S(d) | (S(d+1) - S(d)) << 16
    // at the winner d (each half 0 when that neighbour is outside [0, D)).
    int post;
    const uint8_t* img;   // base image [H][W] (post form)
    int ap2;              // adaptive P2: P2(g) = max(P1, P2 / (1 + g)); else P2
    uint32_t* sub;        // [H][W] (post form, winner-take-all sweeps; optional)
};

// Every sum S held between sweeps fits a byte: with 2 paths S = L_LR <= 31 + P2
// <= 255 always; with 4 paths S = L_LR + L_RL <= 2 * (31 + P2) before the
// vertical pair's winner-take-all (L_r - MC <= P2 from Eq. 3, MC <= 31).
// With the full Census MC <= 62 instead of 31 (mc_max).
inline bool sum_fits_u8(int n_paths, int P2, int mc_max = 31) {
    return (n_paths == 2 && mc_max + P2 <= 255) || (n_paths == 4 && 2 * (mc_max + P2) <= 255);
}

// ---------------------------------------------------------------------------
// Batched execution over device work lists.  A stage of a group of pairs (one
// D, path count, sum width and Census type) is one persistent grid: every
// block takes the next unit of the stage's list (a Census tile, a cost row
// segment, a block of sweep lines, a median tile) with an atomic counter
// until the list is exhausted.  The list lives in device memory: the pairs'
// descriptors in the list's order (longest chains first) and the prefix sums
// of their unit counts.  A kernel skips a descriptor whose D is not its own
// and sets bit 0 of the device status word.
// ---------------------------------------------------------------------------
template <class Job>
struct WorkList {
    const Job* job;         // [n] descriptors
    const uint32_t* start;  // [n + 1]: jobs [0, k) hold units [0, start[k])
    int n;
};

// Features are uint32 (CSCT) or uint64 (full Census) as the launch's ct62 says.
struct CensusJob {
    const uint8_t *left, *right;
    void *Fb, *Fm;
    int W, H;
};
struct CostJob {
    const void *Fb, *Fm;
    uint8_t* rec;  // MC is written at offset 0 of each RB-byte record
    int RB, W, H, D;
};
struct MedianJob {
    const uint8_t* raw;
    uint8_t* out;
    int W, H;
};

// One stage of a group over its work list.
struct ListLaunch {
    const void* list;  // device WorkList<Job> of the stage
    uint32_t* next;    // the list's unit counter, 0 before the launch
    uint32_t* status;  // device status word
    int grid;          // persistent blocks
    int D;
    bool ct62, pair, s8;
    int rx;            // vertical-type sweeps: 0 (vertical, finishing with Eq. 4), +1 / -1 (diagonals)
};

// Each launcher enqueues one kernel on `stream` and returns the launch error.
// ct62 = false: the CSCT of Eq. 1, uint32 features; true: the full 9x7
// Census, uint64 features.
cudaError_t launch_census(const uint8_t* left, const uint8_t* right, void* Fb, void* Fm, int W, int H, bool ct62,
                          cudaStream_t stream);
// MC goes to offset 0 of the RB-byte record of each pixel.
cudaError_t launch_cost(const void* Fb, const void* Fm, uint8_t* rec, int RB, int W, int H, int D, bool ct62,
                        cudaStream_t stream);
cudaError_t launch_sweep_h(const SweepArgs& a, cudaStream_t stream);
// The first sweep stage of a path with pairs (4 or 8 directions): the
// horizontal pair and the first halves (phase 1) of up to three vertical-type
// pairs in one launch; blocks [start[0], start[1]) run the horizontal pair,
// blocks [start[k + 1], start[k + 2]) the first halves of v[k].  `start` is
// filled in by the launcher.
struct FirstStageArgs {
    SweepArgs h;
    SweepArgs v[3];
    int nv;
    int start[5];
};
cudaError_t launch_sweep_first(FirstStageArgs& f, cudaStream_t stream);
// 4 paths: the horizontal first halves (saving their state in f.h.state) beside
// the whole vertical pair f.v[0], which writes S; then the horizontal second
// halves finish with Eq. 4 (launch_sweep_h2, a.state as in the first stage).
cudaError_t launch_sweep_first4(FirstStageArgs& f, cudaStream_t stream);
cudaError_t launch_sweep_h2(const SweepArgs& a, cudaStream_t stream);
cudaError_t launch_sweep_v(const SweepArgs& a, cudaStream_t stream);
// Words of saved path state per vertical-type pair between its two phases:
// per line, 32 lanes x (K + 3) words for each warp carrying it (one warp of
// 16-lane paths, K = D/32; or two warps of 32-lane paths, K = D/64).
inline size_t sweep_state_words(int W, int D) {
    return (D % 64 == 0) ? static_cast<size_t>(W) * 64 * (D / 64 + 3) : static_cast<size_t>(W) * 32 * (D / 32 + 3);
}
cudaError_t launch_median(const uint8_t* raw, uint8_t* disp, int W, int H, cudaStream_t stream);
// Post-filters (sgm_compute_ex).  Mirror: mr[y][x] = right[y][W-1-x],
// ml[y][x] = left[y][W-1-x].
cudaError_t launch_mirror(const uint8_t* left, const uint8_t* right, uint8_t* ml, uint8_t* mr, int W, int H,
                          cudaStream_t stream);
// out16 = 3x3 median of v, v = 16 d + the sub-pixel offset from sub (when
// sub != nullptr) with d = rawL; then, when rawRm != nullptr (the right
// pass's disparity in mirrored columns), 0xFFFF where the left-right check
// fails.
cudaError_t launch_post(const uint8_t* rawL, const uint32_t* sub, const uint8_t* rawRm, uint16_t* out16, int W,
                        int H, int D, cudaStream_t stream);
// The work-list kernels: every job of a list has the launch's D (and, for
// sweeps, its pair / s8 settings; a vertical-type list runs both halves of
// its pair in one unit, the vertical one finishing with Eq. 4).
cudaError_t launch_census_list(const ListLaunch& l, cudaStream_t stream);
cudaError_t launch_cost_list(const ListLaunch& l, cudaStream_t stream);
cudaError_t launch_sweep_h_list(const ListLaunch& l, cudaStream_t stream);
cudaError_t launch_sweep_v_list(const ListLaunch& l, cudaStream_t stream);
cudaError_t launch_median_list(const ListLaunch& l, cudaStream_t stream);
// Units of one pair in each list; blocks of each list kernel resident per SM.
int census_units(int W, int H);
int cost_units(int W, int H);
int sweep_units(int lines, int D, bool pair);
int median_units(int W, int H);
constexpr int kCensusListPerSM = 16, kCostListPerSM = 8, kMedianListPerSM = 8, kSweepListMaxPerSM = 5;
// Debug: paired costs (offset 0 of RB-byte records) -> natural order [H][W][D].
cudaError_t launch_unpair_cost(const uint8_t* rec, int RB, uint8_t* out, int W, int H, int D, cudaStream_t stream);

// ---------------------------------------------------------------------------
// The paired-line 4-path schedule (sgm_pairs.cuh).  Every warp carries two
// adjacent lines of one direction, one per u16 half of each packed word.  The
// per-(pixel, disparity) cubes live in quads of 2 x 2 pixels over the grid
// padded to even sizes W2 x H2: quad (qx, qy) holds, per disparity d, the four
// bytes of pixels (2qx + i, 2qy + j) at byte i + 2j of a 32-bit word, so a
// quad takes QB = 4D bytes of a cube.  Each cube is its own array of
// [QH][QW] quads (FS bytes), at rec + f FS for field f:
//   0 MC    matching costs (Eq. 2); 0 at padding pixels
//   1 LvT   stored L_r of the top-to-bottom path
//   2 LvB   stored L_r of the bottom-to-top path
//   3 Lh0   stored L_r of the left-to-right path
//   4 Lh1   stored L_r of the right-to-left path
// One 32-bit offset q QB then addresses quad q in every field.
// ---------------------------------------------------------------------------
constexpr int kPairsFields = 5;

struct PairsArgs {
    uint8_t* rec;     // the field arrays (kPairsFields of FS bytes each)
    uint8_t* rawq;    // winner-take-all disparity in quads [QH][QW][4]
    uint16_t* Sdbg;   // optional natural-order S [H][W][D] (debug)
    uint32_t* state;  // horizontal chains between the launches: [QH][2][32][K + 1]
    int W, H, W2, H2, QW, QH, D;
    size_t FS;        // bytes of one field array (QH * QW * QB, rounded up)
    int QB;           // bytes of one quad in a field: 4D (W2 * H2 * D < 2^32)
    int n1;           // steps of each horizontal direction in the first launch (even)
    // second launch: left-to-right stores [n1, a) then finishes [a, W2) with
    // Eq. 4; right-to-left stores [b, W2 - n1) then finishes [0, b); columns
    // [b, a) are finished by the parallel winner-take-all
    int a, b;
    uint32_t P1x2, P2x2;
    int s8;           // two stored L_r sum in a byte: 2 (MC_max + P2) <= 255
    int mc_max;       // largest matching cost: 31 (CSCT) or 62 (full Census)
    int nvb, nhb;     // first launch: vertical / horizontal blocks (64 threads each)
    int nh2, npw;     // second launch: chain blocks; parallel winner-take-all blocks (beside them)
    int check_shrink; // bounds-checked build, test hook: bytes taken off the declared end of the fields
};
// Geometry and block counts for a W x H problem (n1 < 0: the default split).
PairsArgs pairs_geometry(int W, int H, int D, int n1);
// Quad-layout matching cost (Eq. 2) into mc: quad q at mc + q QB.
cudaError_t launch_cost_quads(const void* Fb, const void* Fm, uint8_t* mc, int QB, int W, int H, int D, bool ct62,
                              cudaStream_t stream);
cudaError_t launch_pairs_stage1(const PairsArgs& a, cudaStream_t stream);
// The second launch is two kernels that may run side by side: the chains and
// the parallel winner-take-all.
cudaError_t launch_pairs_chain2(const PairsArgs& a, cudaStream_t stream);
cudaError_t launch_pairs_par(const PairsArgs& a, cudaStream_t stream);
// 3x3 median of a quad-layout raw disparity.
cudaError_t launch_median_quads(const uint8_t* rawq, uint8_t* disp, int W, int H, cudaStream_t stream);
// Debug: a quad-layout cube (quad q at cube + q QB) -> natural order [H][W][D].
cudaError_t launch_unquad_cost(const uint8_t* cube, int QB, uint8_t* out, int W, int H, int D, cudaStream_t stream);

bool supported_D(int D);

// One-time kernel attributes; call before any launch or stream capture on the
// current device.
cudaError_t init_kernel_attributes();

}  // namespace sgm
