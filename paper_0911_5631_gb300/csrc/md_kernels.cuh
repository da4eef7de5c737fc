// md_kernels.cuh -- sm_103a kernels of the soft-sphere MD hot path.
//
// One thread per atom (or per cell-ordered slot) throughout, as in the
// paper's GPU formulation (Sec. 2.4: one neighbour column per atom, no use
// of Newton's third law; Sec. 4.2: atom identity from block and thread
// indices).  Included by one translation unit per precision form.
//
// Coordinates.  Every atom belongs to a cell (c_x, c_y, c_z) of width w_d
// (Sec. 2.1).  Its position is the cell centre plus an offset pb (fixed
// between rebuilds, FP32 in the mixed form, FP64 in the FP64 form) plus a
// displacement o (FP64) accumulated since the last rebuild.  The pair
// coordinate every other atom reads is pb + o rounded to the pair precision;
// for a neighbour whose cell lies at offset d (components in {-1, 0, 1},
// periodic wrap included) the separation is (p_i - p_j) - d w, so no
// coordinate of magnitude L ever enters the FP32 arithmetic and |o| is the
// exact displacement used by the skin/2 rebuild rule (Sec. 2.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "md_common.cuh"
#include "md_table.h"

namespace md {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ int64_t gtid() {
    return (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
}

// Set by the last block of a grid to finish, after every other block has
// passed the point of its call.  All threads of the block must call it.
__device__ __forceinline__ bool last_block_done(Counters* C) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int t = atomicAdd(&C->ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// Counters that steer a kernel, read once per block so that every thread of
// the block takes the same branch.
struct View {
    int err;
    int par;
    long long left;
};
__device__ __forceinline__ View load_view(const Counters* C) {
    __shared__ int s_err, s_par;
    __shared__ long long s_left;
    if (threadIdx.x == 0) {
        s_err = C->error;
        s_par = C->parity;
        s_left = C->steps_left;
    }
    __syncthreads();
    return View{s_err, s_par, s_left};
}

// Fixed-shape block sum of kBlock values (result valid in thread 0).
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kBlock / 32; k++) s += sh[k];
    return s;
}

__device__ __forceinline__ int block_max_int(int v, int* sh) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    int s = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kBlock / 32; k++) s = max(s, sh[k]);
    return s;
}

__device__ __forceinline__ void decode_cell(int c, const int G[3], int& cx, int& cy, int& cz) {
    cx = c % G[0];
    int r = c / G[0];
    cy = r % G[1];
    cz = r / G[1];
}

__device__ __forceinline__ int wrap_add(int c, int d, int G) {
    c += d;
    if (c >= G) c -= G;
    if (c < 0) c += G;
    return c;
}

// Shift -d w of a neighbour whose 2-bit cell-offset code is k (d = k - 1).
template <class T>
__device__ __forceinline__ T code_shift(unsigned k, T w) {
    return k == 0u ? w : (k == 2u ? -w : T(0));
}

// Pair coordinate of one component from build offset and displacement.
__device__ __forceinline__ float pair_coord(float pb, double o) { return pb + __double2float_rn(o); }
__device__ __forceinline__ double pair_coord(double pb, double o) { return __dadd_rn(pb, o); }

// FP64 cell-relative offset (build offset + displacement).
__device__ __forceinline__ double full_offset(float pb, double o) { return __dadd_rn((double)pb, o); }
__device__ __forceinline__ double full_offset(double pb, double o) { return __dadd_rn(pb, o); }

// Split an FP64 cell-relative offset t into (pb, o) with pb + o == t.
__device__ __forceinline__ void split_offset(double t, float& pb, double& o) {
    pb = __double2float_rn(t);
    o = __dsub_rn(t, (double)pb);  // exact: pb is t rounded
}
__device__ __forceinline__ void split_offset(double t, double& pb, double& o) {
    pb = t;
    o = 0.0;
}

__device__ __forceinline__ float4 make_pos4(float x, float y, float z, int j) {
    return make_float4(x, y, z, __int_as_float(j));
}
__device__ __forceinline__ double4_32a make_pos4(double x, double y, double z, int j) {
    return make_double4_32a(x, y, z, __longlong_as_double((long long)j));
}
__device__ __forceinline__ int pos4_index(float4 p) { return __float_as_int(p.w); }
__device__ __forceinline__ int pos4_index(double4_32a p) { return (int)__double_as_longlong(p.w); }

__device__ __forceinline__ float4 ld_pos4(const float4* p) { return __ldg(p); }
__device__ __forceinline__ double4_32a ld_pos4(const double4_32a* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return make_double4_32a(a.x, a.y, b.x, b.y);
}

// ---------------------------------------------------------------------------
// pair term, Eq. (1) + shift.  Accumulators per precision form.
// ---------------------------------------------------------------------------

// Mixed form: FP32 pair arithmetic; per-atom sums in int64 fixed point
// (scale 2^32) so the result does not depend on the order of the pairs.
struct AccMixed {
    long long fx = 0, fy = 0, fz = 0, u = 0, w = 0;
    int close = 0;
    __device__ __forceinline__ void pair(const Args<Mixed>& a, float dx, float dy, float dz,
                                         bool energy) {
        float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (r2 < a.rc2f) {
            close |= (r2 < a.close2f);
            float ir2 = __frcp_rn(r2);
            float ir6 = ir2 * ir2 * ir2;
            // 48 * 2^32 is exact in FP32; the scale rides on the force factor
            float frs = (48.0f * kFixScaleF) * ir6 * (ir6 - 0.5f) * ir2;
            fx += __float2ll_rn(frs * dx);
            fy += __float2ll_rn(frs * dy);
            fz += __float2ll_rn(frs * dz);
            if (energy) {
                u += __float2ll_rn(kFixScaleF * fmaf(4.0f * ir6, ir6 - 1.0f, a.ushiftf));
                w += __float2ll_rn(frs * r2);
            }
        }
    }
    __device__ __forceinline__ float force_x() const { return (float)fx * kFixInvF; }
    __device__ __forceinline__ float force_y() const { return (float)fy * kFixInvF; }
    __device__ __forceinline__ float force_z() const { return (float)fz * kFixInvF; }
    __device__ __forceinline__ double energy() const { return (double)u * kFixInv; }
    __device__ __forceinline__ double virial() const { return (double)w * kFixInv; }
};

// FP64 form: everything in double, summed in list order.
struct AccF64 {
    double fx = 0, fy = 0, fz = 0, u = 0, w = 0;
    int close = 0;
    __device__ __forceinline__ void pair(const Args<F64>& a, double dx, double dy, double dz,
                                         bool energy) {
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < a.rc2) {
            close |= (r2 < a.close2);
            double ir2 = 1.0 / r2;
            double ir6 = ir2 * ir2 * ir2;
            double fr = 48.0 * ir6 * (ir6 - 0.5) * ir2;
            fx += fr * dx;
            fy += fr * dy;
            fz += fr * dz;
            if (energy) {
                u += 4.0 * ir6 * (ir6 - 1.0) + a.ushift;
                w += fr * r2;
            }
        }
    }
    __device__ __forceinline__ double force_x() const { return fx; }
    __device__ __forceinline__ double force_y() const { return fy; }
    __device__ __forceinline__ double force_z() const { return fz; }
    __device__ __forceinline__ double energy() const { return u; }
    __device__ __forceinline__ double virial() const { return w; }
};

template <class P> struct AccOf;
template <> struct AccOf<Mixed> { using type = AccMixed; };
template <> struct AccOf<F64> { using type = AccF64; };

// Forces on atom i from its neighbour-list column (Sec. 2.4: W_{m,i}, m_i).
// Entries are read four at a time so several independent loads are in
// flight per thread.
template <class P>
__device__ __forceinline__ void forces_from_list(const Args<P>& a, int i, typename P::real qx,
                                                 typename P::real qy, typename P::real qz,
                                                 const typename P::pos4* __restrict__ pc,
                                                 bool energy, typename AccOf<P>::type& acc) {
    using real = typename P::real;
    using pos4 = typename P::pos4;
    const int cnt = a.nn[i];
    const unsigned nlast = (unsigned)(a.n - 1);  // entries are always < n; the clamp only guards memory
    const int* col = a.nbr + ((size_t)(i >> 5) * (size_t)a.cap) * 32 + (i & 31);
    const real wx = (real)(P::kFp64 ? a.w[0] : a.wf[0]);
    const real wy = (real)(P::kFp64 ? a.w[1] : a.wf[1]);
    const real wz = (real)(P::kFp64 ? a.w[2] : a.wf[2]);
    for (int m = 0; m < cnt; m += 4) {
        unsigned e[4];
        pos4 pj[4];
#pragma unroll
        for (int k = 0; k < 4; k++)
            e[k] = (m + k < cnt) ? (unsigned)__ldcs(col + (size_t)(m + k) * 32) : 0u;
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (m + k < cnt) pj[k] = ld_pos4(pc + min(e[k] & (unsigned)kIndexMask, nlast));
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (m + k < cnt) {
                unsigned code = e[k] >> kCodeShift;
                real dx = (qx - pj[k].x) + code_shift<real>(code & 3u, wx);
                real dy = (qy - pj[k].y) + code_shift<real>((code >> 2) & 3u, wy);
                real dz = (qz - pj[k].z) + code_shift<real>((code >> 4) & 3u, wz);
                acc.pair(a, dx, dy, dz, energy);
            }
        }
    }
}

// Forces on atom i straight from the 27 cells around its cell (cell-list
// only variant; candidates read from the cell-ordered copy).
template <class P>
__device__ __forceinline__ void forces_from_cells(const Args<P>& a, int i, typename P::real qx,
                                                  typename P::real qy, typename P::real qz,
                                                  bool energy, typename AccOf<P>::type& acc) {
    using real = typename P::real;
    using pos4 = typename P::pos4;
    int cx, cy, cz;
    decode_cell(a.cell[i], a.G, cx, cy, cz);
    const real wx = (real)(P::kFp64 ? a.w[0] : a.wf[0]);
    const real wy = (real)(P::kFp64 ? a.w[1] : a.wf[1]);
    const real wz = (real)(P::kFp64 ? a.w[2] : a.wf[2]);
    for (int dz = -1; dz <= 1; dz++) {
        int z = wrap_add(cz, dz, a.G[2]);
        real sz = -(real)dz * wz;
        for (int dy = -1; dy <= 1; dy++) {
            int y = wrap_add(cy, dy, a.G[1]);
            real sy = -(real)dy * wy;
            for (int dx = -1; dx <= 1; dx++) {
                int x = wrap_add(cx, dx, a.G[0]);
                real sx = -(real)dx * wx;
                int c2 = (z * a.G[1] + y) * a.G[0] + x;
                int beg = a.cell_start[c2], end = min(a.cell_start[c2 + 1], (int)a.n);
                for (int t = beg; t < end; t++) {
                    pos4 pj = ld_pos4(a.cand + t);
                    if (pos4_index(pj) == i) continue;
                    acc.pair(a, (qx - pj.x) + sx, (qy - pj.y) + sy, (qz - pj.z) + sz, energy);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// state load
// ---------------------------------------------------------------------------

// Wraps positions into the region, bins them (cell index as defined by
// t = x + L/2, c = floor(t G / L), faces folded back into range) and splits
// the offset from the cell centre into (pb, o).  Storage order = user order.
template <class P>
__global__ void __launch_bounds__(kBlock) k_set_state(Args<P> a) {
    using real = typename P::real;
    using pos4 = typename P::pos4;
    int64_t i = gtid();
    if (i >= a.n) return;
    int c[3];
    real pb[3];
    double o[3];
    bool bad = false;
    for (int d = 0; d < 3; d++) {
        double x = a.io_pos[3 * i + d];
        bad |= !isfinite(x);
        if (!isfinite(x)) x = 0.0;
        double s = floor(__dmul_rn(__dadd_rn(x, a.hL[d]), a.invL[d]));
        x = __dsub_rn(x, __dmul_rn(s, a.L[d]));
        double u = __dadd_rn(x, a.hL[d]);
        int cc = (int)floor(__dmul_rn(u, a.invW[d]));
        if (cc >= a.G[d]) { cc -= a.G[d]; u = __dsub_rn(u, a.L[d]); }
        if (cc < 0) { cc += a.G[d]; u = __dadd_rn(u, a.L[d]); }
        if (cc < 0 || cc >= a.G[d]) {  // only for absurd magnitudes
            bad = true;
            cc = 0;
            u = 0.5 * a.w[d];
        }
        c[d] = cc;
        double t = __dsub_rn(u, __dmul_rn((double)cc + 0.5, a.w[d]));
        split_offset(t, pb[d], o[d]);
        double v = a.io_vel[3 * i + d];
        bad |= !isfinite(v);
    }
    if (bad) atomicOr(&a.ctr->error, kErrUnstable);
    a.cell[i] = (c[2] * a.G[1] + c[1]) * a.G[0] + c[0];
    a.perm[i] = (int)i;
    a.pbx[i] = pb[0]; a.pby[i] = pb[1]; a.pbz[i] = pb[2];
    a.ox[i] = o[0]; a.oy[i] = o[1]; a.oz[i] = o[2];
    a.vx[i] = (typename P::vel)a.io_vel[3 * i + 0];
    a.vy[i] = (typename P::vel)a.io_vel[3 * i + 1];
    a.vz[i] = (typename P::vel)a.io_vel[3 * i + 2];
    a.pA[i] = make_pos4(pair_coord(pb[0], o[0]), pair_coord(pb[1], o[1]), pair_coord(pb[2], o[2]), 0);
}

// Counters for a freshly loaded state: a rebuild with reorder is pending.
template <class P>
__global__ void k_reset_counters(Counters* C) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        Counters z = {};
        z.rebuild_flag = 1;
        z.reorder_now = 1;
        *C = z;
    }
}

template <class P>
__global__ void k_clear_overflow(Counters* C) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        C->error &= ~kErrOverflow;
        C->need_cap = 0;
        C->rebuild_flag = 1;
        C->ticket = 0;
    }
}

// ---------------------------------------------------------------------------
// rebuild: binning (counting sort), reorder, neighbour list
// ---------------------------------------------------------------------------

// Moves each atom whose FP64 offset left its cell into the adjacent cell
// (periodic wrap is an integer operation on the cell coordinate), re-splits
// the offset, refreshes the pair coordinate and counts the cell's atoms.
template <class P>
__global__ void __launch_bounds__(kBlock) k_bin(Args<P> a, int guard) {
    using real = typename P::real;
    using pos4 = typename P::pos4;
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    int64_t i = gtid();
    if (i >= a.n) return;
    int cc[3];
    decode_cell(a.cell[i], a.G, cc[0], cc[1], cc[2]);
    real* pbp[3] = {a.pbx, a.pby, a.pbz};
    double* op[3] = {a.ox, a.oy, a.oz};
    real pb[3];
    double o[3];
    bool bad = false;
    for (int d = 0; d < 3; d++) {
        double t = full_offset(pbp[d][i], op[d][i]);
        for (int it = 0; it < 2; it++) {
            if (t >= a.hw[d]) { t = __dsub_rn(t, a.w[d]); cc[d] = wrap_add(cc[d], 1, a.G[d]); }
            else if (t < -a.hw[d]) { t = __dadd_rn(t, a.w[d]); cc[d] = wrap_add(cc[d], -1, a.G[d]); }
        }
        bad |= !(t >= -a.hw[d] && t < a.hw[d]);  // also catches NaN
        if (!(t >= -a.hw[d] && t < a.hw[d])) t = 0.0;
        split_offset(t, pb[d], o[d]);
        pbp[d][i] = pb[d];
        op[d][i] = o[d];
    }
    if (bad) atomicOr(&C->error, kErrUnstable);
    int c = (cc[2] * a.G[1] + cc[1]) * a.G[0] + cc[0];
    a.cell[i] = c;
    pos4* pc = C->parity ? a.pB : a.pA;
    pc[i] = make_pos4(pair_coord(pb[0], o[0]), pair_coord(pb[1], o[1]), pair_coord(pb[2], o[2]), 0);
    a.rank[i] = atomicAdd(&a.count[c], 1);
}

// Exclusive scan of the cell counts, phase 1: per-tile totals.
template <class P>
__global__ void __launch_bounds__(kBlock) k_scan_tiles(Args<P> a, int guard) {
    __shared__ double sh[kBlock / 32];
    if (guard && !a.ctr->rebuild_flag) return;
    int base = blockIdx.x * kScanTile;
    long long s = 0;
    for (int k = 0; k < kScanTile / kBlock; k++) {
        int c = base + k * kBlock + threadIdx.x;
        if (c < a.ncells) s += a.count[c];
    }
    double t = block_sum((double)s, sh);  // exact: counts are small integers
    if (threadIdx.x == 0) a.tile_sum[blockIdx.x] = (int)t;
}

// Phase 2: one block turns tile totals into exclusive tile offsets.  Also
// resets the per-build maxima.
template <class P>
__global__ void __launch_bounds__(1024) k_scan_top(Args<P> a, int guard) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    if (threadIdx.x == 0) {
        carry = 0;
        C->max_occ = 0;
        C->max_nn = 0;
        C->list_entries = 0;
    }
    __syncthreads();
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < a.ntiles; base += 1024) {
        int idx = base + threadIdx.x;
        int v = idx < a.ntiles ? a.tile_sum[idx] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        int excl = x - v + (warp > 0 ? warp_tot[warp - 1] : 0) + carry;
        if (idx < a.ntiles) a.tile_sum[idx] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
}

// Phase 3: each tile scans its counts from its offset into cell_start and
// records the largest occupancy (the paper's layer count N_l).
template <class P>
__global__ void __launch_bounds__(kBlock) k_scan_apply(Args<P> a, int guard) {
    __shared__ int warp_tot[kBlock / 32];
    __shared__ int shm[kBlock / 32];
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    constexpr int E = kScanTile / kBlock;  // 8 per thread
    int base = blockIdx.x * kScanTile + threadIdx.x * E;
    int v[E];
    int tot = 0, mx = 0;
#pragma unroll
    for (int k = 0; k < E; k++) {
        v[k] = (base + k < a.ncells) ? a.count[base + k] : 0;
        tot += v[k];
        mx = max(mx, v[k]);
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = tot;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    int before = 0;
    for (int k = 0; k < warp; k++) before += warp_tot[k];
    int run = a.tile_sum[blockIdx.x] + before + x - tot;
#pragma unroll
    for (int k = 0; k < E; k++) {
        if (base + k < a.ncells) a.cell_start[base + k] = run;
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.cell_start[a.ncells] = (int)a.n;
    int bm = block_max_int(mx, shm);
    if (threadIdx.x == 0) atomicMax(&C->max_occ, bm);
}

// Places each atom at cell_start[cell] + rank (the cell's arrival order)
// and clears the counts for the next binning.
template <class P>
__global__ void __launch_bounds__(kBlock) k_scatter(Args<P> a, int guard) {
    if (guard && !a.ctr->rebuild_flag) return;
    int64_t lim = a.n > a.ncells ? a.n : a.ncells;
    for (int64_t t = gtid(); t < lim; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < a.n) {
            int slot = a.cell_start[a.cell[t]] + a.rank[t];
            if (slot >= 0 && slot < a.n) a.order[slot] = (int)t;
            else atomicOr(&a.ctr->error, kErrUnstable);
        }
    }
    // counts are no longer needed once cell_start is known
    for (int64_t t = gtid(); t < a.ncells; t += (int64_t)gridDim.x * blockDim.x) a.count[t] = 0;
}

// Makes the order inside each cell deterministic (ascending storage index).
template <class P>
__global__ void __launch_bounds__(kBlock) k_cellsort(Args<P> a, int guard) {
    if (guard && !a.ctr->rebuild_flag) return;
    int64_t c = gtid();
    if (c >= a.ncells) return;
    int beg = a.cell_start[c], end = a.cell_start[c + 1];
    for (int s = beg + 1; s < end; s++) {
        int key = a.order[s];
        int t = s - 1;
        while (t >= beg && a.order[t] > key) {
            a.order[t + 1] = a.order[t];
            t--;
        }
        a.order[t + 1] = key;
    }
}

// Writes the cell-ordered coordinate copy used by the neighbour search and,
// when a reorder is due, the state permuted into cell order (Sec. 2.5).
template <class P>
__global__ void __launch_bounds__(kBlock) k_gather(Args<P> a, int guard) {
    using real = typename P::real;
    using pos4 = typename P::pos4;
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    int64_t s = gtid();
    if (s >= a.n) return;
    const int reorder = C->reorder_now;
    int i = a.order[s];
    real pbx = a.pbx[i], pby = a.pby[i], pbz = a.pbz[i];
    double ox = a.ox[i], oy = a.oy[i], oz = a.oz[i];
    real px = pair_coord(pbx, ox), py = pair_coord(pby, oy), pz = pair_coord(pbz, oz);
    a.cand[s] = make_pos4(px, py, pz, reorder ? (int)s : i);
    if (reorder) {
        a.s_cell[s] = a.cell[i];
        a.s_perm[s] = a.perm[i];
        a.s_pbx[s] = pbx; a.s_pby[s] = pby; a.s_pbz[s] = pbz;
        a.s_ox[s] = ox; a.s_oy[s] = oy; a.s_oz[s] = oz;
        a.s_vx[s] = a.vx[i]; a.s_vy[s] = a.vy[i]; a.s_vz[s] = a.vz[i];
    }
}

// Copies the permuted state back (only when a reorder is due).
template <class P>
__global__ void __launch_bounds__(kBlock) k_commit(Args<P> a, int guard) {
    using pos4 = typename P::pos4;
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    if (!C->reorder_now) return;
    int64_t s = gtid();
    if (s >= a.n) return;
    a.cell[s] = a.s_cell[s];
    a.perm[s] = a.s_perm[s];
    a.pbx[s] = a.s_pbx[s]; a.pby[s] = a.s_pby[s]; a.pbz[s] = a.s_pbz[s];
    a.ox[s] = a.s_ox[s]; a.oy[s] = a.s_oy[s]; a.oz[s] = a.s_oz[s];
    a.vx[s] = a.s_vx[s]; a.vy[s] = a.s_vy[s]; a.vz[s] = a.s_vz[s];
    pos4 p = a.cand[s];
    pos4* pc = C->parity ? a.pB : a.pA;
    pc[s] = p;
}

// Exact FP64 neighbour criterion r^2 < r_n^2 on the cell-relative offsets
// (no contraction, fixed operation order).
template <class P>
__device__ __forceinline__ bool within_rn_fp64(const Args<P>& a, int i, int j, int dx, int dy, int dz) {
    double ex = __dadd_rn(__dsub_rn(full_offset(a.pbx[i], a.ox[i]), full_offset(a.pbx[j], a.ox[j])),
                          __dmul_rn(-(double)dx, a.w[0]));
    double ey = __dadd_rn(__dsub_rn(full_offset(a.pby[i], a.oy[i]), full_offset(a.pby[j], a.oy[j])),
                          __dmul_rn(-(double)dy, a.w[1]));
    double ez = __dadd_rn(__dsub_rn(full_offset(a.pbz[i], a.oz[i]), full_offset(a.pbz[j], a.oz[j])),
                          __dmul_rn(-(double)dz, a.w[2]));
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    return r2 < a.rn2;
}

// Neighbour-list build (Sec. 2.4): for the atom in cell-ordered slot s, scan
// the 27 cells around its cell and record every j != i with r < r_n in its
// column together with the cell-offset code.  The decision is the FP64
// criterion; the mixed form evaluates it only for candidates whose FP32
// distance falls in a narrow band around r_n.
template <class P>
__global__ void __launch_bounds__(kBlock) k_build(Args<P> a, int guard) {
    using real = typename P::real;
    using pos4 = typename P::pos4;
    __shared__ int shm[kBlock / 32];
    __shared__ double shs[kBlock / 32];
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    int64_t s = gtid();
    int m = 0;
    if (s < a.n) {
        pos4 ci = a.cand[s];
        int i = pos4_index(ci);
        int cx, cy, cz;
        decode_cell(a.cell[i], a.G, cx, cy, cz);
        int* col = a.nbr + ((size_t)(i >> 5) * (size_t)a.cap) * 32 + (i & 31);
        for (int dz = -1; dz <= 1; dz++) {
            int z = wrap_add(cz, dz, a.G[2]);
            for (int dy = -1; dy <= 1; dy++) {
                int y = wrap_add(cy, dy, a.G[1]);
                for (int dx = -1; dx <= 1; dx++) {
                    int x = wrap_add(cx, dx, a.G[0]);
                    int c2 = (z * a.G[1] + y) * a.G[0] + x;
                    unsigned code = (unsigned)(dx + 1) | ((unsigned)(dy + 1) << 2) | ((unsigned)(dz + 1) << 4);
                    int beg = a.cell_start[c2], end = min(a.cell_start[c2 + 1], (int)a.n);
                    if constexpr (P::kFp64) {
                        double sx = __dmul_rn(-(double)dx, a.w[0]);
                        double sy = __dmul_rn(-(double)dy, a.w[1]);
                        double sz = __dmul_rn(-(double)dz, a.w[2]);
                        for (int t = beg; t < end; t++) {
                            if (t == s) continue;
                            pos4 pj = ld_pos4(a.cand + t);
                            double ex = __dadd_rn(__dsub_rn((double)ci.x, (double)pj.x), sx);
                            double ey = __dadd_rn(__dsub_rn((double)ci.y, (double)pj.y), sy);
                            double ez = __dadd_rn(__dsub_rn((double)ci.z, (double)pj.z), sz);
                            double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                            if (r2 < a.rn2) {
                                if (m < a.cap) col[(size_t)m * 32] = pos4_index(pj) | (int)(code << kCodeShift);
                                m++;
                            }
                        }
                    } else {
                        float sx = -(float)dx * a.wf[0];
                        float sy = -(float)dy * a.wf[1];
                        float sz = -(float)dz * a.wf[2];
                        for (int t = beg; t < end; t++) {
                            if (t == s) continue;
                            pos4 pj = ld_pos4(a.cand + t);
                            float ex = ((float)ci.x - (float)pj.x) + sx;
                            float ey = ((float)ci.y - (float)pj.y) + sy;
                            float ez = ((float)ci.z - (float)pj.z) + sz;
                            float r2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                            bool take = r2 < a.rn2_lo;
                            if (!take && r2 < a.rn2_hi) take = within_rn_fp64(a, i, pos4_index(pj), dx, dy, dz);
                            if (take) {
                                if (m < a.cap) col[(size_t)m * 32] = pos4_index(pj) | (int)(code << kCodeShift);
                                m++;
                            }
                        }
                    }
                }
            }
        }
        a.nn[i] = m < a.cap ? m : a.cap;
        if (m > a.cap) {
            atomicOr(&C->error, kErrOverflow);
            atomicMax(&C->need_cap, m);
        }
    }
    int bm = block_max_int(m, shm);
    double bs = block_sum((double)m, shs);
    if (threadIdx.x == 0) {
        atomicMax(&C->max_nn, bm);
        atomicAdd((unsigned long long*)&C->list_entries, (unsigned long long)bs);
    }
}

// Closes a rebuild: counters, reorder bookkeeping, flag cleared.
template <class P>
__global__ void k_rebuild_done(Args<P> a, int guard) {
    Counters* C = a.ctr;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (guard && !C->rebuild_flag) return;
    C->rebuilds += 1;
    if (C->reorder_now) {
        C->reorders += 1;
        C->since_reorder = 0;
        C->reorder_now = 0;
    }
    C->rebuild_flag = 0;
}

// Graph prologue: copies the device rebuild flag into the first
// conditional node's handle.
template <class P>
__global__ void k_cond(Args<P> a, cudaGraphConditionalHandle h) {
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, a.ctr->rebuild_flag ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// integration
// ---------------------------------------------------------------------------

// Rebuild decision at the end of a drift: list invalid once some atom has
// moved skin/2 (every step in the cell-list-only variant); reorder when
// reorder_interval steps have passed (Sec. 5.4).
__device__ __forceinline__ int decide_rebuild(Counters* C, int cell_list_only, int interval) {
    int need = (C->far_flag != 0u) || cell_list_only;
    C->far_flag = 0u;
    C->rebuild_flag = need;
    C->reorder_now = need && interval > 0 && C->since_reorder >= interval;
    return need;
}

// First half of the first step of an md_step call (Sec. 2.1 (a)): half kick
// with the stored forces, drift, displacement test.
template <class P>
__global__ void __launch_bounds__(kBlock) k_kickdrift(Args<P> a, long long nsteps) {
    using real = typename P::real;
    using vel = typename P::vel;
    using pos4 = typename P::pos4;
    Counters* C = a.ctr;
    const View vw = load_view(C);
    const int err = vw.err;
    const int par = vw.par;
    int64_t i = gtid();
    bool far = false;
    if (!err && i < a.n) {
        pos4* pc = par ? a.pB : a.pA;
        vel vx = a.vx[i], vy = a.vy[i], vz = a.vz[i];
        double ox = a.ox[i], oy = a.oy[i], oz = a.oz[i];
        if constexpr (P::kFp64) {
            vx = fma((double)a.h, (double)a.fx[i], (double)vx);
            vy = fma((double)a.h, (double)a.fy[i], (double)vy);
            vz = fma((double)a.h, (double)a.fz[i], (double)vz);
        } else {
            vx = fmaf(a.hf, (float)a.fx[i], (float)vx);
            vy = fmaf(a.hf, (float)a.fy[i], (float)vy);
            vz = fmaf(a.hf, (float)a.fz[i], (float)vz);
        }
        ox = fma((double)vx, a.dt, ox);
        oy = fma((double)vy, a.dt, oy);
        oz = fma((double)vz, a.dt, oz);
        real px = pair_coord(a.pbx[i], ox), py = pair_coord(a.pby[i], oy), pz = pair_coord(a.pbz[i], oz);
        a.vx[i] = vx; a.vy[i] = vy; a.vz[i] = vz;
        a.ox[i] = ox; a.oy[i] = oy; a.oz[i] = oz;
        pc[i] = make_pos4(px, py, pz, 0);
        if constexpr (P::kFp64) far = ox * ox + oy * oy + oz * oz >= a.thr2;
        else {
            float fx = __double2float_rn(ox), fy = __double2float_rn(oy), fz = __double2float_rn(oz);
            far = fmaf(fx, fx, fmaf(fy, fy, fz * fz)) >= a.thr2f;
        }
    }
    if (__any_sync(0xffffffffu, far) && (threadIdx.x & 31) == 0) atomicOr(&C->far_flag, 1u);
    if (last_block_done(C)) {
        if (threadIdx.x == 0) {
            if (!err) {
                C->steps_left = nsteps;
                decide_rebuild(C, a.cell_list_only, a.reorder_interval);
            }
            C->ticket = 0;
        }
    }
}

// Force + integration kernel (Sec. 2.1 (c)-(e) of one step and (a) of the
// next).  Mode kModeInit computes the forces of a freshly loaded state.
// Mode kModeAuto completes a step: forces f_n, v_n = v_{n-1/2} + f_n dt/2;
// then, unless it is the last step of the call, v_{n+1/2} = v_n + f_n dt/2,
// o += v_{n+1/2} dt into the other pair-coordinate buffer and the skin/2
// test.  The last block advances the counters and, in a graph, sets the
// next conditional rebuild node.
template <class P, bool kCells>
__global__ void __launch_bounds__(kBlock) k_step(Args<P> a, int mode, cudaGraphConditionalHandle next,
                                                 int has_next) {
    using real = typename P::real;
    using vel = typename P::vel;
    using pos4 = typename P::pos4;
    __shared__ double shs[kBlock / 32];
    Counters* C = a.ctr;
    const View vw = load_view(C);
    const int err = vw.err;
    const long long left = vw.left;
    const int par = vw.par;
    const bool init = (mode == kModeInit);
    const bool active = init || (err == 0 && left > 0);
    const bool last = !init && left == 1;
    const bool energy = init || last;
    const pos4* pc = par ? a.pB : a.pA;
    pos4* pn = par ? a.pA : a.pB;
    int64_t i = gtid();
    bool far = false, close = false;
    double ke = 0.0, pe = 0.0, vir = 0.0;
    if (active && i < a.n) {
        real pbx = a.pbx[i], pby = a.pby[i], pbz = a.pbz[i];
        double ox = a.ox[i], oy = a.oy[i], oz = a.oz[i];
        real qx = pair_coord(pbx, ox), qy = pair_coord(pby, oy), qz = pair_coord(pbz, oz);
        typename AccOf<P>::type acc;
        if (kCells) forces_from_cells<P>(a, (int)i, qx, qy, qz, energy, acc);
        else forces_from_list<P>(a, (int)i, qx, qy, qz, pc, energy, acc);
        close = acc.close != 0;
        real fx = acc.force_x(), fy = acc.force_y(), fz = acc.force_z();
        vel vx = a.vx[i], vy = a.vy[i], vz = a.vz[i];
        if (!init) {
            if constexpr (P::kFp64) {
                vx = fma((double)a.h, (double)fx, (double)vx);
                vy = fma((double)a.h, (double)fy, (double)vy);
                vz = fma((double)a.h, (double)fz, (double)vz);
            } else {
                vx = fmaf(a.hf, (float)fx, (float)vx);
                vy = fmaf(a.hf, (float)fy, (float)vy);
                vz = fmaf(a.hf, (float)fz, (float)vz);
            }
        }
        if (energy) {
            a.fx[i] = fx; a.fy[i] = fy; a.fz[i] = fz;
            double dvx = vx, dvy = vy, dvz = vz;
            ke = 0.5 * (dvx * dvx + dvy * dvy + dvz * dvz);
            pe = 0.5 * acc.energy();
            vir = 0.5 * acc.virial();
            if (!init) { a.vx[i] = vx; a.vy[i] = vy; a.vz[i] = vz; }
        } else {
            if constexpr (P::kFp64) {
                vx = fma((double)a.h, (double)fx, (double)vx);
                vy = fma((double)a.h, (double)fy, (double)vy);
                vz = fma((double)a.h, (double)fz, (double)vz);
            } else {
                vx = fmaf(a.hf, (float)fx, (float)vx);
                vy = fmaf(a.hf, (float)fy, (float)vy);
                vz = fmaf(a.hf, (float)fz, (float)vz);
            }
            ox = fma((double)vx, a.dt, ox);
            oy = fma((double)vy, a.dt, oy);
            oz = fma((double)vz, a.dt, oz);
            a.vx[i] = vx; a.vy[i] = vy; a.vz[i] = vz;
            a.ox[i] = ox; a.oy[i] = oy; a.oz[i] = oz;
            pn[i] = make_pos4(pair_coord(pbx, ox), pair_coord(pby, oy), pair_coord(pbz, oz), 0);
            if constexpr (P::kFp64) far = ox * ox + oy * oy + oz * oz >= a.thr2;
            else {
                float dx = __double2float_rn(ox), dy = __double2float_rn(oy), dz = __double2float_rn(oz);
                far = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= a.thr2f;
            }
        }
    }
    if (__any_sync(0xffffffffu, far) && (threadIdx.x & 31) == 0) atomicOr(&C->far_flag, 1u);
    if (__any_sync(0xffffffffu, close) && (threadIdx.x & 31) == 0) atomicOr(&C->close_flag, 1);
    if (energy && active) {
        double bk = block_sum(ke, shs);
        double bp = block_sum(pe, shs);
        double bw = block_sum(vir, shs);
        if (threadIdx.x == 0) {
            a.part[3 * blockIdx.x + 0] = bk;
            a.part[3 * blockIdx.x + 1] = bp;
            a.part[3 * blockIdx.x + 2] = bw;
        }
    }
    if (last_block_done(C)) {
        if (threadIdx.x == 0) {
            int need = 0;
            if (!init && err == 0 && left > 0) {
                C->steps_left = left - 1;
                C->step += 1;
                C->since_reorder += 1;
                if (!last) {
                    C->parity = par ^ 1;
                    need = decide_rebuild(C, a.cell_list_only, a.reorder_interval);
                } else {
                    C->far_flag = 0u;
                    C->rebuild_flag = 0;
                }
            } else if (!init) {
                C->far_flag = 0u;
            }
            if (C->close_flag) {
                C->error |= kErrClose;
                C->close_flag = 0;
            }
            if (has_next) cudaGraphSetConditional(next, need ? 1u : 0u);
            C->ticket = 0;
        }
    }
}

// Sums the per-block partials of the last init/final step in a fixed order.
template <class P>
__global__ void __launch_bounds__(kBlock) k_finalize(Args<P> a) {
    __shared__ double shs[kBlock / 32];
    double s[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < a.nblocks; b += kBlock)
        for (int k = 0; k < 3; k++) s[k] += a.part[3 * b + k];
    double t0 = block_sum(s[0], shs);
    double t1 = block_sum(s[1], shs);
    double t2 = block_sum(s[2], shs);
    if (threadIdx.x == 0) {
        a.ctr->ke = t0;
        a.ctr->pe = t1;
        a.ctr->virial = t2;
    }
}

// ---------------------------------------------------------------------------
// state export (user order)
// ---------------------------------------------------------------------------

template <class P>
__global__ void __launch_bounds__(kBlock) k_get_state(Args<P> a) {
    int64_t i = gtid();
    if (i >= a.n) return;
    int u = a.perm[i];
    int cc[3];
    decode_cell(a.cell[i], a.G, cc[0], cc[1], cc[2]);
    const typename P::real* pb[3] = {a.pbx, a.pby, a.pbz};
    const double* o[3] = {a.ox, a.oy, a.oz};
    const typename P::vel* v[3] = {a.vx, a.vy, a.vz};
    for (int d = 0; d < 3; d++) {
        double centre = __dsub_rn(__dmul_rn((double)cc[d] + 0.5, a.w[d]), a.hL[d]);
        double x = __dadd_rn(centre, full_offset(pb[d][i], o[d][i]));
        double s = floor(__dmul_rn(__dadd_rn(x, a.hL[d]), a.invL[d]));
        x = __dsub_rn(x, __dmul_rn(s, a.L[d]));
        a.io_pos[3 * (int64_t)u + d] = x;
        a.io_vel[3 * (int64_t)u + d] = (double)v[d][i];
    }
}

template <class P>
__global__ void __launch_bounds__(kBlock) k_get_forces(Args<P> a, double* out) {
    int64_t i = gtid();
    if (i >= a.n) return;
    int64_t u = a.perm[i];
    out[3 * u + 0] = (double)a.fx[i];
    out[3 * u + 1] = (double)a.fy[i];
    out[3 * u + 2] = (double)a.fz[i];
}

template <class P>
__global__ void __launch_bounds__(kBlock) k_get_cells(Args<P> a, int* out) {
    int64_t i = gtid();
    if (i >= a.n) return;
    out[a.perm[i]] = a.cell[i];
}

// ---------------------------------------------------------------------------
// kernel table used by the host runtime (graph nodes and eager launches)
// ---------------------------------------------------------------------------

template <class P>
KernelTable<P> make_kernel_table() {
    KernelTable<P> t;
    t.set_state = (void*)k_set_state<P>;
    t.bin = (void*)k_bin<P>;
    t.scan_tiles = (void*)k_scan_tiles<P>;
    t.scan_top = (void*)k_scan_top<P>;
    t.scan_apply = (void*)k_scan_apply<P>;
    t.scatter = (void*)k_scatter<P>;
    t.cellsort = (void*)k_cellsort<P>;
    t.gather = (void*)k_gather<P>;
    t.commit = (void*)k_commit<P>;
    t.build = (void*)k_build<P>;
    t.rebuild_done = (void*)k_rebuild_done<P>;
    t.cond = (void*)k_cond<P>;
    t.kickdrift = (void*)k_kickdrift<P>;
    t.step_list = (void*)k_step<P, false>;
    t.step_cells = (void*)k_step<P, true>;
    t.finalize = (void*)k_finalize<P>;
    t.get_state = (void*)k_get_state<P>;
    t.get_forces = (void*)k_get_forces<P>;
    t.get_cells = (void*)k_get_cells<P>;
    t.reset_counters = (void*)k_reset_counters<P>;
    t.clear_overflow = (void*)k_clear_overflow<P>;
    return t;
}

}  // namespace md
