// md_common.cuh -- device-state layout shared by the kernels and the host
// runtime of libmd.  Internal; the public interface is include/md.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace md {

// Threads per block for every per-atom / per-slot kernel.
constexpr int kBlock = 256;
// Threads per block of the mixed form's plain step kernel (with a neighbour
// list): 128 measured about 2 % faster than 256 at the 1M-atom workload.
// The final step of a call, which writes per-block energy partials, keeps
// kBlock.
constexpr int kStepBlockMixed = 128;
// The step's closing work (counters, rebuild decision, next conditional
// node) runs as a one-warp kernel after the step kernel rather than in the
// step kernel's last block.
constexpr bool kStepTailNode = true;
// Each warp of the step kernel reads the counters itself (no opening block
// barrier).
constexpr bool kWarpView = true;
// A graph evaluates the rebuild condition (a conditional node, about 5 us
// whether taken or not) before every kRebuildEvery-th step only; a step in
// between whose rebuild is due waits (does nothing) for the next one, and
// the call runs the waited steps at its end.  A waiting step still launches
// its grid, whose cost grows with the system: measured, checking every third
// step gains 5 % at 1M atoms and loses 1 % at 8M, so systems above
// kRebuildEveryMaxAtoms check before every step.
constexpr int kRebuildEvery = 3;
constexpr int64_t kRebuildEveryMaxAtoms = int64_t(1) << 21;
constexpr int kStageRows = 12;  // neighbour-list rows a step-kernel warp copies to shared memory
// The force loop reads the staged rows four at a time (the reads are not
// predicated, only the gathers they feed), so the staged count -- the
// smaller of kStageRows and the list capacity, itself rounded up to a
// multiple of 4 -- must be a multiple of 4 to stay inside the warp's rows.
static_assert(kStageRows % 4 == 0, "kStageRows must be a multiple of 4");
// The skin shell [r_c, r_n) is cut into kShellBins bins of width skin /
// kShellBins.  The build sorts each atom's entries by the bin of their
// distance at the build and records, for k = 1 .. kShellBins, how many
// entries lie below r_c + k skin / kShellBins; a step then reads only the
// entries that the displacements since the build can have brought inside
// r_c.  The build stages up to kBuildStage candidates per atom in shared
// memory.
constexpr int kShellBins = 8;
constexpr int kBuildStage = 18;
// The build's bin counts sit in the bytes of one 64-bit word: eight bins,
// and no count above 255.
static_assert(kShellBins == 8 && kBuildStage < 256, "one byte per shell bin in a 64-bit word");
// Threads per block of the thread-per-atom build (its stage: kBuildStage
// 8-byte words per thread in shared memory; 18 measured best at the 1M-atom
// workload, against 16, 20, 24 and 32).
constexpr int kBuildBlock = 128;
// The build's candidate loop issues kBuildUnroll loads before it uses them,
// and the cell ranges of the next (c_y, c_z) row are loaded while a row runs.
constexpr int kBuildUnroll = 4;
constexpr bool kBuildPrefetch = true;
// The grid kernels keep the running maximum of the squared displacement in
// kD2Buckets words, one per 128-byte line (block b uses word b mod
// kD2Buckets), so that the atomics of the many warps of a launch do not
// queue at one address.
constexpr int kD2Buckets = 64;
// Dynamic shared memory of the ensemble engine, ints per thread: the larger
// of the step's staged rows and the build's staging (entries and distances).
// The engine's build stages kEnsBuildStage candidates per atom: a deeper
// stage leaves its 1024-thread blocks less L1 for the step phase, a shallower
// one sends too many atoms of its denser replicas to the rescan (measured
// at the 512-replica workload: 16 beats 12, 14, 20 and 24).
constexpr int kEnsBuildStage = 16;
static_assert(kEnsBuildStage < 256, "one byte per shell bin in a 64-bit word");
constexpr int kEnsSmemInts = kStageRows > 2 * kEnsBuildStage ? kStageRows : 2 * kEnsBuildStage;
// Elements per block of the cell-count scan (kBlock threads x 8).
constexpr int kScanTile = 2048;
// Largest neighbour capacity of the mixed form (its fixed-point partial
// sums stay inside int32 for up to this many terms).
constexpr int kMaxCapMixed = 512;
// Neighbour entries are j | code << kCodeShift; code packs the cell offset
// (d_x+1) | (d_y+1) << 2 | (d_z+1) << 4 of j's cell relative to i's cell, the
// periodic-image information beta of Sec. 3.2 in 6 high bits.
constexpr int kCodeShift = 26;
constexpr int kIndexMask = (1 << kCodeShift) - 1;
constexpr int64_t kMaxAtoms = int64_t(1) << kCodeShift;
// Fixed-point scale of the mixed form's per-atom sums.
constexpr double kFixScale = 4294967296.0;       // 2^32
constexpr float kFixScaleF = 4294967296.0f;
constexpr float kFixInvF = 2.3283064365386963e-10f;  // 2^-32
constexpr double kFixInv = 2.3283064365386963e-10;

// Error bits recorded on the device.
enum : int {
    kErrOverflow = 1,   // neighbour list longer than its capacity
    kErrUnstable = 2,   // non-finite coordinate or velocity
    kErrClose = 4,      // pair closer than the fixed-point range allows
    kErrInternal = 8,   // a plain step node met the last step of a call
};

// Step-kernel modes.
enum : int {
    kModeInit = 0,  // forces of the loaded state; velocities untouched
    kModeAuto = 1,  // a full step, or the final half-kick when one step is left
};

// Counters and flags kept on the device (one per handle).
struct Counters {
    int error;                 // kErr* bits
    int need_cap;              // largest neighbour count seen by an overflowing build
    int rebuild_flag;          // the next rebuild branch must run
    int reorder_now;           // the pending rebuild also reorders the atoms
    int parity;                // which pair-coordinate buffer is current (0 = A)
    int max_nn;                // largest neighbour count at the last build
    int max_occ;               // largest cell occupancy at the last binning
    unsigned int ticket;       // last-block-done counter (reset by the last block)
    unsigned int far_flag;     // some atom moved skin/2 since the last build
    int close_flag;            // a pair came too close during the running step
    unsigned int d2max;        // bits of the largest squared displacement (FP32, >= 0)
                               // seen since the last build: a running maximum
    int reach;                 // shell reach of the next step (1..kShellBins)
    long long steps_left;      // steps still to run in the current md_step
    long long step;            // steps completed since the state was loaded
    long long since_reorder;   // steps since the last reorder
    long long rebuilds;        // rebuilds since the state was loaded
    long long reorders;        // reorders since the state was loaded
    long long list_entries;    // neighbour-list length at the last build
    long long list_reads;      // entries the profiled steps read (k_count_reads)
    // reduced measurement of the last finalize
    double ke, pe, virial;
};

// One job of an ensemble launch: replica `rep` (index into the Args array);
// load its state first when `init`; then advance it `nsteps` steps.
struct EnsJob {
    int rep;
    int init;
    long long nsteps;
    unsigned long long t_start, t_end;  // device clock (ns) around the job's work
};

// Precision forms.  real: pair arithmetic, build offsets and saved forces;
// vel: velocity storage; pos4: gathered coordinates (x, y, z, payload).
struct Mixed {
    using real = float;
    using vel = float;
    using pos4 = float4;
    static constexpr bool kFp64 = false;
};
struct F64 {
    using real = double;
    using vel = double;
    using pos4 = double4_32a;
    static constexpr bool kFp64 = true;
};

// Everything the kernels need, passed by value.  Device pointers only.
template <class P>
struct alignas(16) Args {
    using real = typename P::real;
    using vel = typename P::vel;
    using pos4 = typename P::pos4;

    int64_t n;          // atoms
    int cap;            // neighbour slots per atom
    int ncells;
    int G[3];
    int ntiles;         // scan tiles
    int nblocks;        // ceil(n / kBlock)
    int cell_list_only;
    int reorder_interval;
    int shell_bins;     // lists sorted by shell bin, steps read up to the shell reach
    int list_rows;      // list layout: 0 = a warp's 32 columns interleaved, 1 = each atom's entries contiguous

    double L[3], hL[3], invL[3], invW[3];
    double w[3];        // cell widths
    double hw[3];       // half cell widths
    float hwf_in[3];    // FP32 bound below which an offset is surely inside its cell
    unsigned jmask;     // pair_slots(n) - 1: masks a list entry to its index (below n for every
                        // entry a build writes) and keeps any masked index inside pA / pB
    double hw_in[3];    // FP64 bound below which the whole-cell moves of a re-binning are exact
    float wf[3];
    double dt, h;       // time step and half step
    float dtf, hf;
    double rc2;         // r_c^2
    float rc2f;
    double rn2;         // r_n^2
    float rn2_lo, rn2_hi;  // FP32 pre-filter band around r_n^2
    double ushift;
    float ushiftf;
    double thr2;        // (skin/2)^2
    float thr2f;
    float close2f;      // pairs closer than this flag kErrClose
    float fix_small_fr; // mixed form: a pair with f/r below this has every force component under 2^11
    float rcf;          // r_c
    float shell_inv;    // kShellBins / skin (0 without a skin)
    float shell_eps;    // rounding margin of the shell-bin bound (distance units)
    double close2;

    // per-atom state, storage order
    int* cell;          // cell index of the last binning
    int* perm;          // storage index -> user id
    int* rank;          // arrival rank within the cell (binning scratch)
    real* pbx; real* pby; real* pbz;   // cell-relative offset at the last build
    double* ox; double* oy; double* oz; // displacement since the last build
    vel* vx; vel* vy; vel* vz;
    real* fx; real* fy; real* fz;      // forces of the last completed step
    pos4* pA; pos4* pB;                // current cell-relative coordinates (ping-pong), pair_slots(n) each
    float4* cand;                      // FP32 coordinates in cell order + storage index

    // reorder scratch (same shapes as the state)
    int* s_cell; int* s_perm;
    real* s_pbx; real* s_pby; real* s_pbz;
    double* s_ox; double* s_oy; double* s_oz;
    vel* s_vx; vel* s_vy; vel* s_vz;

    // cells
    int* count;         // [ncells] atoms per cell (kept zero between binnings)
    int* cell_start;    // [ncells + 1]
    int* order;         // [n] storage index of each cell-ordered slot
    int* tile_sum;      // [ntiles] then exclusive tile offsets

    // neighbour list: entry m of atom i at ((i / 32) * cap + m) * 32 + i % 32
    int* nbr;
    int* nn;            // [n] entries per atom
    unsigned char* lim; // [kShellBins - 1][n] entries to read at shell reach k = 1..7 in
                        // plane k - 1; 255 = all (nn)
    unsigned* d2b;      // [kD2Buckets * 32] running maxima (grid kernels; word 32 b);
                        // null: ctr->d2max alone (the ensemble engine)

    double* part;       // [3 * nblocks] per-block KE, PE, W
    Counters* ctr;

    double* io_pos;     // [3 n] staging for set/get (user order, AoS)
    double* io_vel;     // [3 n]
};

// Slots of each pair-coordinate buffer: n rounded up to a power of two, so
// that the force loop's gather index, an entry masked with jmask =
// pair_slots(n) - 1, stays inside the buffer whatever the entry holds (a
// clamp to n - 1 would cost the loop one more integer instruction per
// entry).  No entry a build writes has an index of n or more.
__host__ __device__ __forceinline__ int64_t pair_slots(int64_t n) {
    int64_t s = 1;
    while (s < n) s <<= 1;
    return s;
}

// Entry m of atom i's neighbour list (Sec. 3.4, W_{m,i}) sits at
// list_base(i) + m list_stride: by default the columns of a warp's 32 atoms
// are interleaved, ((i / 32) cap + m) 32 + i % 32, so that a warp reading
// row m of its atoms touches one 128-byte line; with list_rows each atom's
// entries are contiguous, i cap + m (the paper's W transposed).
template <class P>
__host__ __device__ __forceinline__ size_t list_base(const Args<P>& a, int64_t i) {
    return a.list_rows ? (size_t)i * (size_t)a.cap : ((size_t)(i >> 5) * (size_t)a.cap) * 32 + (size_t)(i & 31);
}
template <class P>
__host__ __device__ __forceinline__ int list_stride(const Args<P>& a) {
    return a.list_rows ? 1 : 32;
}

// x slices of the pencil cell order (tiles of 4 x 4 cells in (y, z), each
// taken at every c_x): the thread blocks of the warp-cooperative build.
constexpr int kWcThreads = 512;  // one warp per cell of a slice
template <class P>
__host__ __device__ __forceinline__ int64_t wc_slices(const Args<P>& a) {
    return (int64_t)((a.G[1] + 3) / 4) * ((a.G[2] + 3) / 4) * a.G[0];
}

}  // namespace md
