// md_kernels.cuh -- sm_103a kernels of the soft-sphere MD hot path.
//
// One thread per atom (or per cell-ordered slot) throughout, as in the
// paper's GPU formulation (Sec. 3.4: one neighbour column per atom, no use
// of Newton's third law; Sec. 4.2: atom identity from block and thread
// indices).  Included by one translation unit per precision form.
//
// Coordinates.  Every atom belongs to a cell (c_x, c_y, c_z) of width w_d
// (Sec. 3.1).  Its position is the cell centre plus an offset pb (fixed
// between rebuilds, FP32 in the mixed form, FP64 in the FP64 form) plus a
// displacement o (FP64) accumulated since the last rebuild.  The pair
// coordinate every other atom reads is pb + o rounded to the pair precision;
// for a neighbour whose cell lies at offset d (components in {-1, 0, 1},
// periodic wrap included) the separation is (p_i - p_j) - d w, so no
// coordinate of magnitude L ever enters the FP32 arithmetic and |o| is the
// exact displacement used by the skin/2 rebuild rule (Sec. 3.1).
//
// GB300 note.  The FP64 pipe issues about two instructions per clock per SM
// here, and so do the hardware conversions float<->int64 and
// double<->float.  The mixed form therefore keeps FP64 to the three
// position-update FMAs per atom and step, and does most of its conversions
// on the FP32 and integer pipes (namespace cvt, struct Fix); the step
// kernel, whose integer pipe is the busiest, converts the displacement to
// FP32 on the FP64 pipe instead.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include "md_common.cuh"
#include "md_table.h"

namespace md {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ int64_t gtid() {
    return (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
}

// True in the last block of the grid to get here, after every other block
// has passed the same point.  All threads of the block must call it.
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
// Asynchronous 16-byte global->shared copy (L2 only) and the wait for all
// of this thread's outstanding copies.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// pend: a rebuild is due and has not run (the step's list is stale).
struct View {
    int err;
    int par;
    long long left;
    int pend;
};
// The same view read by each warp on its own (lane 0 reads, a shuffle
// spreads it): no block barrier.
__device__ __forceinline__ View load_view_warp(const Counters* C) {
    int e = 0, p = 0, r = 0;
    long long l = 0;
    if ((threadIdx.x & 31) == 0) {
        e = C->error;
        p = C->parity;
        l = C->steps_left;
        r = C->rebuild_flag;
    }
    return View{__shfl_sync(0xffffffffu, e, 0), __shfl_sync(0xffffffffu, p, 0), __shfl_sync(0xffffffffu, l, 0),
                __shfl_sync(0xffffffffu, r, 0)};
}
__device__ __forceinline__ View load_view(const Counters* C) {
    __shared__ int s_err, s_par, s_pend;
    __shared__ long long s_left;
    if (threadIdx.x == 0) {
        s_err = C->error;
        s_par = C->parity;
        s_left = C->steps_left;
        s_pend = C->rebuild_flag;
    }
    __syncthreads();
    return View{s_err, s_par, s_left, s_pend};
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

// Cell coordinates are stored packed, 10 bits each (G_d <= 1023).
__device__ __forceinline__ int pack_cell(int cx, int cy, int cz) { return cx | (cy << 10) | (cz << 20); }
__device__ __forceinline__ void unpack_cell(int p, int& cx, int& cy, int& cz) {
    cx = p & 1023;
    cy = (p >> 10) & 1023;
    cz = (p >> 20) & 1023;
}
// Scalar cell index c = (c_z G_y + c_y) G_x + c_x (0-based form of Sec. 3.1),
// the cell id reported to callers.
__device__ __forceinline__ int linear_cell(int cx, int cy, int cz, const int G[3]) {
    return (cz * G[1] + cy) * G[0] + cx;
}
__device__ __forceinline__ int linear_of_packed(int p, const int G[3]) {
    int cx, cy, cz;
    unpack_cell(p, cx, cy, cz);
    return linear_cell(cx, cy, cz, G);
}

// Storage order of the cells: the order of count, cell_start and of every
// cell-ordered array.  Sec. 3.5 only asks that the atoms of a cell sit
// together; which cell comes next is free.  Here the (y, z) cross-section is
// cut into tiles of 4 x 4 cells (narrower at the high faces), each tile
// extended along x is a pencil, pencils follow one another tile row by tile
// row, and a pencil lists its cells one x slice after the other.  A thread
// block's atoms then fill a few slices of one pencil, so they and their
// 27-cell neighbourhoods span a few kilobytes and the neighbour reads of the
// force and build kernels mostly hit in L1.  For fixed (c_y, c_z) the index
// is base + c_x * stride.
struct PencilRow {
    int base, stride;
};
__device__ __forceinline__ PencilRow pencil_row(int cy, int cz, const int G[3]) {
    const int y0 = cy & ~3, z0 = cz & ~3;
    const int hy = min(4, G[1] - y0), hz = min(4, G[2] - z0);
    PencilRow r;
    r.stride = hy * hz;
    r.base = (z0 * G[1] + y0 * hz) * G[0] + (cz - z0) * hy + (cy - y0);
    return r;
}
__device__ __forceinline__ int cell_index(int cx, int cy, int cz, const int G[3]) {
    const PencilRow r = pencil_row(cy, cz, G);
    return r.base + cx * r.stride;
}
__device__ __forceinline__ int cell_index_of_packed(int p, const int G[3]) {
    int cx, cy, cz;
    unpack_cell(p, cx, cy, cz);
    return cell_index(cx, cy, cz, G);
}

__device__ __forceinline__ int wrap_add(int c, int d, int G) {
    c += d;
    if (c >= G) c -= G;
    if (c < 0) c += G;
    return c;
}

// ---------------------------------------------------------------------------
// absolute coordinates and the cell rule of Sec. 3.2 / Sec. 4.2
// ---------------------------------------------------------------------------
//
// The position of an atom is defined as the FP64 number abs_coord(c, t) of
// each component: the centre of its cell, (c + 1/2) w - L/2, plus the
// cell-relative offset t, wrapped into [-L/2, L/2) by x - L floor((x + L/2)/L).
// md_get_state reports exactly these numbers.  The cell of a wrapped
// coordinate x is floor((x + L/2) G/L), folded into [0, G) (Sec. 4.2
// truncates (r + L/2) / w the same way).  Every binning decides a cell by
// this rule on the reported position, and the offset relative to the new
// cell is x - centre, which is exact whenever x and the centre are within a
// factor of two of each other (then abs_coord gives back x itself).  So
// cell_of(md_get_state positions) equals the stored cells, element by
// element, as the FP64 reference computes it.

__device__ __forceinline__ double cell_centre(int c, double w, double hL) {
    return __dsub_rn(__dmul_rn((double)c + 0.5, w), hL);
}

template <class P>
__device__ __forceinline__ double abs_coord(const Args<P>& a, int d, int c, double t) {
    const double x = __dadd_rn(cell_centre(c, a.w[d], a.hL[d]), t);
    const double s = floor(__dmul_rn(__dadd_rn(x, a.hL[d]), a.invL[d]));
    return __dsub_rn(x, __dmul_rn(s, a.L[d]));
}

// Cell of the wrapped coordinate x and its offset from that cell's centre.
// An x that rounds onto the upper face belongs to cell 0 (and one below the
// lower face to cell G - 1); its offset is then taken from the periodic
// image next to that cell.  Returns false (cell 0, offset 0) for a
// non-finite x and for a magnitude too large to have been wrapped.
template <class P>
__device__ __forceinline__ bool bin_coord(const Args<P>& a, int d, double x, int& c, double& t) {
    if (!isfinite(x)) {
        c = 0;
        t = 0.0;
        return false;
    }
    const double q = floor(__dmul_rn(__dadd_rn(x, a.hL[d]), a.invW[d]));
    if (!(q >= -1.0 && q <= (double)a.G[d])) {  // a wrapped x gives q in [0, G]
        c = 0;
        t = 0.0;
        return false;
    }
    c = (int)q;
    double xe = x;
    if (c >= a.G[d]) { c -= a.G[d]; xe = __dsub_rn(x, a.L[d]); }
    if (c < 0) { c += a.G[d]; xe = __dadd_rn(x, a.L[d]); }
    t = __dsub_rn(xe, cell_centre(c, a.w[d], a.hL[d]));
    return true;
}

// Shift -d w of a neighbour whose 2-bit cell-offset code is k (d = k - 1).
template <class T>
__device__ __forceinline__ T code_shift(unsigned k, T w) {
    return k == 0u ? w : (k == 2u ? -w : T(0));
}

// ---------------------------------------------------------------------------
// Conversions on the FP32 and integer pipes.  They follow the IEEE 754
// binary32/binary64 encodings with round-to-nearest-even; values below the
// binary32 normal range are flushed to signed zero, which the coordinates
// and forces here never reach.  md_selftest compares them with the hardware
// conversions.
// ---------------------------------------------------------------------------
namespace cvt {

// binary32 -> binary64 (exact).
__device__ __forceinline__ double f64(float x) {
    unsigned b = __float_as_uint(x);
    unsigned s = b & 0x80000000u;
    unsigned e = (b >> 23) & 0xFFu;
    unsigned m = b & 0x7FFFFFu;
    unsigned hi = s | ((e + 896u) << 20) | (m >> 3);
    unsigned lo = m << 29;
    if (e == 0u) { hi = s; lo = 0u; }
    if (e == 255u) hi = s | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u);
    return __hiloint2double((int)hi, (int)lo);
}

// binary64 -> binary32, round to nearest, ties to even.
__device__ __forceinline__ float f32(double x) {
    unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    unsigned s = hi & 0x80000000u;
    int E = (int)((hi >> 20) & 0x7FFu);
    int e = E - 896;
    unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    unsigned rest = lo & 0x1FFFFFFFu;
    unsigned f = s | ((unsigned)e << 23) | m;
    f += (unsigned)((rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u)));
    if (e <= 0) f = s;
    if (e >= 255) f = s | 0x7F800000u | ((E == 0x7FF && ((hi & 0xFFFFFu) | lo)) ? 0x400000u : 0u);
    return __uint_as_float(f);
}

// int64 -> binary32, round to nearest, ties to even.
__device__ __forceinline__ float from_fix(long long q) {
    unsigned long long mag = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
    if (mag == 0ull) return 0.0f;
    int lz = __clzll((long long)mag);
    unsigned long long nrm = mag << lz;
    unsigned m = (unsigned)(nrm >> 40);
    unsigned long long rest = nrm & 0xFFFFFFFFFFull;
    unsigned f = ((unsigned)(190 - lz) << 23) + (m & 0x7FFFFFu);
    f += (unsigned)((rest > 0x8000000000ull) | ((rest == 0x8000000000ull) & (m & 1u)));
    return __uint_as_float(f | (q < 0 ? 0x80000000u : 0u));
}

}  // namespace cvt

// Fixed point with scale 2^32 kept as three int32 partial sums.
// add(g) adds round(g 2^32) (ties to even) for |g| < 2^30 as
// a 2^44 + b 2^22 + c with |a| <= 2^18, |b|, |c| <= 2^21: each chunk is
// rounded to an integer by the magic-number method -- adding 1.5 2^23 in
// FP32 round-to-nearest leaves round(x) in the low mantissa bits for
// |x| < 2^22, so the integer is the bit pattern minus that of 1.5 2^23 (the
// float-to-integer conversion of C. Hecker, "Let's Get to the (Floating)
// Point", Game Developer, 1996) -- and every remainder is exact, so the
// three sums are exact and independent of the order of the terms, and
// add(-g) subtracts exactly what add(g) adds.  value()
// assembles the int64 sum.  With at most 512 terms no partial sum leaves
// int32.  For |g| <= 2^11 the first chunk is zero and its remainder is g
// itself, so add_small(g) -- the last two chunks alone -- adds exactly
// what add(g) adds.
constexpr float kFixMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kFixMagicBits = 0x4B400000;  // its bit pattern
constexpr float kFixSmall = 2048.0f;       // add_small is exact up to this magnitude
struct Fix {
    int a = 0, b = 0, c = 0;
    __device__ __forceinline__ void add_small(float g) {
        float s2 = fmaf(g, 1024.0f, kFixMagic);
        b += __float_as_int(s2) - kFixMagicBits;
        float r2 = fmaf(s2 - kFixMagic, -0x1p-10f, g);
        float s3 = fmaf(r2, 4294967296.0f, kFixMagic);
        c += __float_as_int(s3) - kFixMagicBits;
    }
    __device__ __forceinline__ void add(float g) {
        float s1 = fmaf(g, 0x1p-12f, kFixMagic);
        a += __float_as_int(s1) - kFixMagicBits;
        add_small(fmaf(s1 - kFixMagic, -4096.0f, g));
    }
    __device__ __forceinline__ long long value() const {
        return (long long)a * (1ll << 44) + (long long)b * (1ll << 22) + (long long)c;
    }
};

// Two binary32 values in one 64-bit register pair, for the packed FP32
// instructions (add/sub/mul/fma .f32x2) of sm_100-class GPUs: one issue
// slot computes both halves, each rounded exactly as the scalar
// instruction would.  The first value sits in the low half.
struct F2 {
    unsigned long long v;
};
__device__ __forceinline__ F2 f2(float x, float y) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ void f2_get(F2 p, float& x, float& y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(p.v));
}
__device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(x.v), "l"(y.v));
    return r;
}
__device__ __forceinline__ F2 f2_sub(F2 x, F2 y) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(x.v), "l"(y.v));
    return r;
}
__device__ __forceinline__ F2 f2_mul(F2 x, F2 y) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(x.v), "l"(y.v));
    return r;
}
__device__ __forceinline__ F2 f2_fma(F2 x, F2 y, F2 z) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(x.v), "l"(y.v), "l"(z.v));
    return r;
}

// Two Fix sums advanced together with the packed instructions (the same
// operations, so the same integers, as two Fix::add_small calls).
struct Fix2 {
    Fix x, y;
    __device__ __forceinline__ void add_small(F2 g) {
        const F2 M = f2(kFixMagic, kFixMagic);
        float lo, hi;
        F2 s2 = f2_fma(g, f2(1024.0f, 1024.0f), M);
        f2_get(s2, lo, hi);
        x.b += __float_as_int(lo) - kFixMagicBits;
        y.b += __float_as_int(hi) - kFixMagicBits;
        F2 r2 = f2_fma(f2_sub(s2, M), f2(-0x1p-10f, -0x1p-10f), g);
        F2 s3 = f2_fma(r2, f2(4294967296.0f, 4294967296.0f), M);
        f2_get(s3, lo, hi);
        x.c += __float_as_int(lo) - kFixMagicBits;
        y.c += __float_as_int(hi) - kFixMagicBits;
    }
};

// Pair coordinate of one component from build offset and displacement.
__device__ __forceinline__ float pair_coord(float pb, double o) { return pb + cvt::f32(o); }
__device__ __forceinline__ double pair_coord(double pb, double o) { return __dadd_rn(pb, o); }

// FP64 cell-relative offset (build offset + displacement).
__device__ __forceinline__ double full_offset(float pb, double o) { return __dadd_rn(cvt::f64(pb), o); }
__device__ __forceinline__ double full_offset(double pb, double o) { return __dadd_rn(pb, o); }

// Split an FP64 cell-relative offset t into (pb, o) with pb + o == t.
__device__ __forceinline__ void split_offset(double t, float& pb, double& o) {
    pb = cvt::f32(t);
    o = __dsub_rn(t, cvt::f64(pb));  // exact: pb is t rounded
}
__device__ __forceinline__ void split_offset(double t, double& pb, double& o) {
    pb = t;
    o = 0.0;
}

// Drift of one displacement component: o += v dt in FP64.
__device__ __forceinline__ double drift(double o, float v, double dt) { return fma(cvt::f64(v), dt, o); }
__device__ __forceinline__ double drift(double o, double v, double dt) { return fma(v, dt, o); }

// Pair coordinate after a drift and the squared displacement in the pair
// precision (the skin/2 test).
// kHw: the hardware conversion (on the FP64 pipe) instead of the bit-level
// one (integer pipe), the same round-to-nearest result.  The grid step
// kernel, whose integer pipe is its busiest, takes the hardware one; the
// ensemble engine, whose 1024-thread blocks load the FP64 pipe more, the
// bit-level one (measured: each choice is the faster one for its kernel).
template <bool kHw = false>
__device__ __forceinline__ float moved(float pb, double o, float& p) {
    float d;
    if constexpr (kHw) d = __double2float_rn(o);
    else d = cvt::f32(o);
    p = pb + d;
    return d * d;
}
template <bool kHw = false>
__device__ __forceinline__ double moved(double pb, double o, double& p) {
    p = __dadd_rn(pb, o);
    return o * o;
}

__device__ __forceinline__ float4 make_pos4(float x, float y, float z, int j) {
    return make_float4(x, y, z, __int_as_float(j));
}
__device__ __forceinline__ double4_32a make_pos4(double x, double y, double z, int j) {
    return make_double4_32a(x, y, z, __longlong_as_double((long long)j));
}
__device__ __forceinline__ float4 ld_pos4(const float4* p) { return __ldg(p); }
__device__ __forceinline__ double4_32a ld_pos4(const double4_32a* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return make_double4_32a(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(double x) { return cvt::f32(x); }

// ---------------------------------------------------------------------------
// pair term, Eq. (1) + shift, and the per-atom accumulators
// ---------------------------------------------------------------------------

// Mixed form: FP32 pair arithmetic; per-atom sums in int64 fixed point.
// The x and y components travel as packed pairs.  A pair term whose
// components all stay within kFixSmall (|f r| < kFixSmall / r_c bounds
// them, which holds for every r above about 0.75) skips the first,
// all-zero chunk.
struct AccMixed {
    Fix2 fxy;
    Fix fz, u, w;
    int close = 0;
    // accumulate one interacting pair (r^2 < r_c^2) at separation d
    template <bool kEnergy>
    __device__ __forceinline__ void force(const Args<Mixed>& a, F2 dxy, float dz, float r2) {
        float ir2 = __fdividef(1.0f, r2);
        float ir6 = ir2 * ir2 * ir2;
        float fr = 48.0f * ir6 * (ir6 - 0.5f) * ir2;
        F2 gxy = f2_mul(f2(fr, fr), dxy);
        float gz = fr * dz;
        if (fr < a.fix_small_fr) {
            fxy.add_small(gxy);
            fz.add_small(gz);
        } else {
            // a pair closer than sqrt(close2f) has f/r far above
            // fix_small_fr, so the close test belongs to this branch only
            close |= (r2 < a.close2f);
            float gx, gy;
            f2_get(gxy, gx, gy);
            fxy.x.add(gx);
            fxy.y.add(gy);
            fz.add(gz);
        }
        if constexpr (kEnergy) {
            u.add(fmaf(4.0f * ir6, ir6 - 1.0f, a.ushiftf));
            w.add(fr * r2);
        }
    }
    template <bool kEnergy>
    __device__ __forceinline__ void force(const Args<Mixed>& a, float dx, float dy, float dz, float r2) {
        force<kEnergy>(a, f2(dx, dy), dz, r2);
    }
    __device__ __forceinline__ float r2(float dx, float dy, float dz) const { return fmaf(dx, dx, fmaf(dy, dy, dz * dz)); }
    __device__ __forceinline__ bool inside(const Args<Mixed>& a, float r2) const { return r2 < a.rc2f; }
    template <bool kEnergy>
    __device__ __forceinline__ void pair(const Args<Mixed>& a, float dx, float dy, float dz) {
        float rr = r2(dx, dy, dz);
        if (inside(a, rr)) force<kEnergy>(a, f2(dx, dy), dz, rr);
    }
    // Per-atom force from the three exact partial sums.  The rounding is
    // not the correctly rounded one, but it is a fixed function of sums
    // that do not depend on the order of the pairs.
    __device__ __forceinline__ static float to_force(const Fix& q) {
        return fmaf((float)q.a, 4096.0f, fmaf((float)q.b, 0x1p-10f, (float)q.c * 0x1p-32f));
    }
    __device__ __forceinline__ float force_x() const { return to_force(fxy.x); }
    __device__ __forceinline__ float force_y() const { return to_force(fxy.y); }
    __device__ __forceinline__ float force_z() const { return to_force(fz); }
    __device__ __forceinline__ double energy() const { return (double)u.value() * kFixInv; }
    __device__ __forceinline__ double virial() const { return (double)w.value() * kFixInv; }
};

// FP64 form: everything in double, summed in list order.
struct AccF64 {
    double fx = 0, fy = 0, fz = 0, u = 0, w = 0;
    int close = 0;
    template <bool kEnergy>
    __device__ __forceinline__ void force(const Args<F64>& a, double dx, double dy, double dz, double r2) {
        close |= (r2 < a.close2);
        double ir2 = 1.0 / r2;
        double ir6 = ir2 * ir2 * ir2;
        double fr = 48.0 * ir6 * (ir6 - 0.5) * ir2;
        fx += fr * dx;
        fy += fr * dy;
        fz += fr * dz;
        if constexpr (kEnergy) {
            u += 4.0 * ir6 * (ir6 - 1.0) + a.ushift;
            w += fr * r2;
        }
    }
    __device__ __forceinline__ double r2(double dx, double dy, double dz) const { return dx * dx + dy * dy + dz * dz; }
    __device__ __forceinline__ bool inside(const Args<F64>& a, double r2) const { return r2 < a.rc2; }
    template <bool kEnergy>
    __device__ __forceinline__ void pair(const Args<F64>& a, double dx, double dy, double dz) {
        double rr = r2(dx, dy, dz);
        if (inside(a, rr)) force<kEnergy>(a, dx, dy, dz, rr);
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

// Per-thread queue of interacting pairs (separation, r^2) in shared memory,
// slot-major so that a warp's accesses are contiguous.
template <class P> struct Queue;
template <> struct Queue<Mixed> {
    using item = float4;
    static constexpr int kSlots = 6;
    __device__ __forceinline__ static item make(float x, float y, float z, float r2) { return make_float4(x, y, z, r2); }
};
template <> struct Queue<F64> {
    using item = double4_32a;
    static constexpr int kSlots = 3;
    __device__ __forceinline__ static item make(double x, double y, double z, double r2) {
        return make_double4_32a(x, y, z, r2);
    }
};

// Shift -d w for each 6-bit cell-offset code, built per block in shared
// memory (entries whose code has a component 3 are unused).
template <class P>
__device__ __forceinline__ void fill_shift_table(const Args<P>& a, typename P::pos4* tbl) {
    using real = typename P::real;
    if (threadIdx.x < 64) {
        unsigned c = threadIdx.x;
        real w0, w1, w2;
        if constexpr (P::kFp64) { w0 = a.w[0]; w1 = a.w[1]; w2 = a.w[2]; }
        else { w0 = a.wf[0]; w1 = a.wf[1]; w2 = a.wf[2]; }
        tbl[c] = make_pos4(code_shift<real>(c & 3u, w0), code_shift<real>((c >> 2) & 3u, w1),
                           code_shift<real>((c >> 4) & 3u, w2), 0);
    }
}

// Forces on atom i from its neighbour-list column (Sec. 3.4: W_{m,i}, m_i),
// in two phases.  Phase 1 reads the entries (four at a time, so several
// independent loads are in flight), tests r^2 < r_c^2 and queues the
// interacting separations; phase 2 evaluates the pair term for the queued
// pairs only.  A warp thus runs the expensive pair term as often as its
// busiest atom has interacting partners instead of as often as it has
// neighbour entries.  Pairs beyond the queue are evaluated at once.  The
// first `staged` rows of the warp's column block are already in shared
// memory (rows), the rest is read from global memory.
template <class P, bool kEnergy>
__device__ __forceinline__ void forces_from_list(const Args<P>& a, int cnt, const int* col, const int* rows, int staged,
                                                 typename P::real qx, typename P::real qy, typename P::real qz,
                                                 const typename P::pos4* __restrict__ pc,
                                                 const typename P::pos4* __restrict__ shift,
                                                 typename Queue<P>::item* queue,
                                                 typename AccOf<P>::type& acc) {
    using real = typename P::real;
    using pos4 = typename P::pos4;
    constexpr int kQ = Queue<P>::kSlots;
    const unsigned jmask = a.jmask;  // entries are always < n; the mask only guards memory
    int nq = 0;
    for (int m = 0; m < cnt; m += 4) {
        unsigned e[4];
        pos4 pj[4];
#pragma unroll
        for (int k = 0; k < 4; k++)
            e[k] = (m + k < cnt) ? (unsigned)(m + k < staged ? rows[(m + k) * 32 + (threadIdx.x & 31)]
                                                             : __ldcs(col + (size_t)(m + k) * 32))
                                 : 0u;
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (m + k < cnt) pj[k] = ld_pos4(pc + (e[k] & jmask));
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (m + k < cnt) {
                const pos4 sh = shift[e[k] >> kCodeShift];
                real dx = (qx - pj[k].x) + sh.x;
                real dy = (qy - pj[k].y) + sh.y;
                real dz = (qz - pj[k].z) + sh.z;
                real rr = acc.r2(dx, dy, dz);
                if (acc.inside(a, rr)) {
                    if (nq < kQ) queue[nq * blockDim.x + threadIdx.x] = Queue<P>::make(dx, dy, dz, rr);
                    else acc.template force<kEnergy>(a, dx, dy, dz, rr);
                    nq++;
                }
            }
        }
    }
    const int nk = min(nq, kQ);
    for (int k = 0; k < nk; k++) {
        const auto d = queue[k * blockDim.x + threadIdx.x];
        acc.template force<kEnergy>(a, d.x, d.y, d.z, d.w);
    }
}

// Mixed-form counterpart of forces_from_list, in one pass: each entry's
// pair term is evaluated as soon as its distance test passes.  Here the
// shared-memory queue and the shift table cost more L1 data-pipe
// wavefronts than the divergence they save, so the shift
// -d w = (1 - k) w of each component (k the 2-bit code) is computed from
// the code, and the staged rows and the rest of the column run as two loops
// (no per-entry choice of source).  x and y travel as one packed pair.
__device__ __forceinline__ float small_int_to_float(unsigned k) {  // exact for k < 2^22
    return __uint_as_float(0x4B400000u | k) - 12582912.0f;
}
// A gathered pair coordinate: through the read-only path (the paper's
// texture cache, Sec. 4.4) or, for the ablation, a plain coherent load.
template <bool kLdg>
__device__ __forceinline__ float4 gather4(const float4* p) {
    if constexpr (kLdg) {
        return __ldg(p);
    } else {
        float4 v;
        asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "l"(p));
        return v;
    }
}

template <bool kEnergy, bool kLdg = true, bool kRows = false>
__device__ __forceinline__ void forces_mixed(const Args<Mixed>& a, int cnt, const int* col, const int* rows,
                                             int staged, float qx, float qy, float qz,
                                             const float4* __restrict__ pc, AccMixed& acc) {
    const unsigned jmask = a.jmask;  // entries are always < n; the mask only guards memory
    const int lane = threadIdx.x & 31;
    const F2 qxy = f2(qx, qy);
    const F2 wxy = f2(a.wf[0], a.wf[1]);
    const F2 nwxy = f2(-a.wf[0], -a.wf[1]);
    const float wz = a.wf[2];
    const float rc2 = a.rc2f;
    auto pair = [&](unsigned e, const float4& pj) {
        const unsigned c = e >> kCodeShift;
        const F2 kxy = f2(small_int_to_float(c & 3u), small_int_to_float((c >> 2) & 3u));
        const F2 sxy = f2_fma(kxy, nwxy, wxy);  // (1 - k) w, exact
        const float sz = fmaf(small_int_to_float(c >> 4), -wz, wz);
        const F2 dxy = f2_add(f2_sub(qxy, f2(pj.x, pj.y)), sxy);
        const float dz = (qz - pj.z) + sz;
        float sx, sy;
        f2_get(f2_mul(dxy, dxy), sx, sy);
        const float rr = fmaf(dz, dz, sx + sy);
        if (rr < rc2) acc.template force<kEnergy>(a, dxy, dz, rr);
    };
    const int ns = min(cnt, staged);  // staged is a multiple of 4 or the capacity
    int m = 0;
    for (; m < ns; m += 4) {
        unsigned e[4];
        float4 pj[4];
#pragma unroll
        for (int k = 0; k < 4; k++) e[k] = (unsigned)rows[(m + k) * 32 + lane];  // rows past ns are unused
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (m + k < ns) pj[k] = gather4<kLdg>(pc + (e[k] & jmask));
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (m + k < ns) pair(e[k], pj[k]);
    }
    constexpr int kStride = kRows ? 1 : 32;
    for (m = ns; m < cnt; m += 4) {
        unsigned e[4];
        float4 pj[4];
#pragma unroll
        for (int k = 0; k < 4; k++) e[k] = (m + k < cnt) ? (unsigned)__ldcs(col + (size_t)(m + k) * kStride) : 0u;
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (m + k < cnt) pj[k] = gather4<kLdg>(pc + (e[k] & jmask));
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (m + k < cnt) pair(e[k], pj[k]);
    }
}

// Forces on atom i straight from the 27 cells around its cell (cell-list
// only variant).  Candidates come from the cell-ordered copy; their pair
// coordinates are read from the current buffer (FP64 form) or the copy
// itself (mixed form, where the two hold the same numbers).
template <class P, bool kEnergy>
__device__ __forceinline__ void forces_from_cells(const Args<P>& a, int i, typename P::real qx,
                                                  typename P::real qy, typename P::real qz,
                                                  const typename P::pos4* __restrict__ pc,
                                                  typename AccOf<P>::type& acc) {
    using real = typename P::real;
    int cx, cy, cz;
    unpack_cell(a.cell[i], cx, cy, cz);
    real wx, wy, wz;
    if constexpr (P::kFp64) { wx = a.w[0]; wy = a.w[1]; wz = a.w[2]; }
    else { wx = a.wf[0]; wy = a.wf[1]; wz = a.wf[2]; }
    for (int dz = -1; dz <= 1; dz++) {
        int z = wrap_add(cz, dz, a.G[2]);
        real sz = -(real)dz * wz;
        for (int dy = -1; dy <= 1; dy++) {
            int y = wrap_add(cy, dy, a.G[1]);
            real sy = -(real)dy * wy;
            for (int dx = -1; dx <= 1; dx++) {
                int x = wrap_add(cx, dx, a.G[0]);
                real sx = -(real)dx * wx;
                int c2 = cell_index(x, y, z, a.G);
                int beg = a.cell_start[c2], end = min(a.cell_start[c2 + 1], (int)a.n);
                for (int t = beg; t < end; t++) {
                    float4 cj = __ldg(a.cand + t);
                    int j = __float_as_int(cj.w);
                    if (j == i) continue;
                    real px, py, pz;
                    if constexpr (P::kFp64) {
                        auto pj = ld_pos4(pc + min((unsigned)j, (unsigned)(a.n - 1)));
                        px = pj.x; py = pj.y; pz = pj.z;
                    } else {
                        px = cj.x; py = cj.y; pz = cj.z;
                    }
                    acc.template pair<kEnergy>(a, (qx - px) + sx, (qy - py) + sy, (qz - pz) + sz);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// state load
// ---------------------------------------------------------------------------

// Wraps positions into the region, bins them by the cell rule above and
// splits the offset from the cell centre into (pb, o).  Storage order = user
// order.
template <class P>
__device__ __forceinline__ void set_state_item(const Args<P>& a, int64_t i) {
    using real = typename P::real;
    int c[3];
    real pb[3];
    double o[3];
    bool bad = false;
    for (int d = 0; d < 3; d++) {
        double x = a.io_pos[3 * i + d];
        bad |= !isfinite(x);
        if (!isfinite(x)) x = 0.0;
        const double s = floor(__dmul_rn(__dadd_rn(x, a.hL[d]), a.invL[d]));
        x = __dsub_rn(x, __dmul_rn(s, a.L[d]));
        double t;
        bad |= !bin_coord(a, d, x, c[d], t);
        split_offset(t, pb[d], o[d]);
        double v = a.io_vel[3 * i + d];
        bad |= !isfinite(v);
    }
    if (bad) atomicOr(&a.ctr->error, kErrUnstable);
    a.cell[i] = pack_cell(c[0], c[1], c[2]);
    a.perm[i] = (int)i;
    a.pbx[i] = pb[0]; a.pby[i] = pb[1]; a.pbz[i] = pb[2];
    a.ox[i] = o[0]; a.oy[i] = o[1]; a.oz[i] = o[2];
    if constexpr (P::kFp64) {
        a.vx[i] = a.io_vel[3 * i + 0];
        a.vy[i] = a.io_vel[3 * i + 1];
        a.vz[i] = a.io_vel[3 * i + 2];
    } else {
        a.vx[i] = cvt::f32(a.io_vel[3 * i + 0]);
        a.vy[i] = cvt::f32(a.io_vel[3 * i + 1]);
        a.vz[i] = cvt::f32(a.io_vel[3 * i + 2]);
    }
    a.pA[i] = make_pos4(pair_coord(pb[0], o[0]), pair_coord(pb[1], o[1]), pair_coord(pb[2], o[2]), 0);
}

template <class P>
__global__ void __launch_bounds__(kBlock) k_set_state(Args<P> a) {
    using real = typename P::real;
    int64_t i = gtid();
    if (i >= a.n) return;
    set_state_item<P>(a, i);
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

// Re-anchors every atom at its current position: the FP64 offset pb + o
// becomes the new build offset (o restarts from the rounding remainder), and
// an atom whose offset left its cell moves to the cell the rule above gives
// for the position md_get_state reports (periodic wrap is an integer
// operation on the cell coordinate).  Refreshes the pair coordinate and
// counts the atoms of each cell.
template <class P>
__device__ __forceinline__ int bin_item(const Args<P>& a, int64_t i) {
    using real = typename P::real;
    Counters* C = a.ctr;
    int cc[3];
    unpack_cell(a.cell[i], cc[0], cc[1], cc[2]);
    real* pbp[3] = {a.pbx, a.pby, a.pbz};
    double* op[3] = {a.ox, a.oy, a.oz};
    real pb[3];
    double o[3];
    bool bad = false;
    for (int d = 0; d < 3; d++) {
        const double t = full_offset(pbp[d][i], op[d][i]);
        split_offset(t, pb[d], o[d]);
        // An offset clearly inside the cell keeps it (the rule gives the same
        // cell with a margin of 1e-6 w); NaN fails the test.  Otherwise the
        // atom moves by whole cells while its offset lies outside
        // [-w/2, w/2), which is what the rule decides as long as the new
        // offset stays 1e-9 w/2 or more inside the faces (the rounding of the
        // rule is below 1e-13 w for any region of up to 10^5 cells); an
        // offset closer to a face, or an atom more than two cells away, is
        // binned by the rule itself from the reported position.
        if (!(fabsf(to_f32(pb[d])) < a.hwf_in[d])) {
            double tn = t;
            int c = cc[d];
            for (int it = 0; it < 2; it++) {
                if (tn >= a.hw[d]) { tn = __dsub_rn(tn, a.w[d]); c = wrap_add(c, 1, a.G[d]); }
                else if (tn < -a.hw[d]) { tn = __dadd_rn(tn, a.w[d]); c = wrap_add(c, -1, a.G[d]); }
            }
            if (!(fabs(tn) < a.hw_in[d])) bad |= !bin_coord(a, d, abs_coord(a, d, cc[d], t), c, tn);
            cc[d] = c;
            split_offset(tn, pb[d], o[d]);
        }
        pbp[d][i] = pb[d];
        op[d][i] = o[d];
    }
    if (bad) atomicOr(&C->error, kErrUnstable);
    a.cell[i] = pack_cell(cc[0], cc[1], cc[2]);
    typename P::pos4* pc = C->parity ? a.pB : a.pA;
    pc[i] = make_pos4(pair_coord(pb[0], o[0]), pair_coord(pb[1], o[1]), pair_coord(pb[2], o[2]), 0);
    const int c = cell_index(cc[0], cc[1], cc[2], a.G);
    a.rank[i] = atomicAdd(&a.count[c], 1);
    return c;
}

// Binning of every atom, and phase 1 of the exclusive scan of the cell
// counts: the atoms of each scan tile (kScanTile consecutive cells) are
// added to its total, one atomic per tile present in a warp (a warp's atoms
// are mostly in one tile).  Also resets the per-build maxima.
template <class P>
__global__ void __launch_bounds__(kBlock) k_bin(Args<P> a, int guard) {
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        C->max_occ = 0;
        C->max_nn = 0;
        C->list_entries = 0;
    }
    const int64_t i = gtid();
    const int tile = i < a.n ? bin_item<P>(a, i) / kScanTile : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, tile);
    if (tile >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&a.tile_sum[tile], __popc(peers));
}

// Phase 2: each tile adds up the totals of the tiles below it (its offset),
// scans its counts from there into cell_start and records the largest
// occupancy (the paper's layer count N_l).
template <class P>
__global__ void __launch_bounds__(kBlock) k_scan_apply(Args<P> a, int guard) {
    __shared__ int warp_tot[kBlock / 32];
    __shared__ int shm[kBlock / 32];
    __shared__ int s_pre[kBlock / 32];
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    {
        int pre = 0;
        for (int t = threadIdx.x; t < (int)blockIdx.x; t += kBlock) pre += a.tile_sum[t];
        for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
        if ((threadIdx.x & 31) == 0) s_pre[threadIdx.x >> 5] = pre;
    }
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
    for (int k = 0; k < kBlock / 32; k++) before += s_pre[k];
    int run = before + x - tot;
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
__device__ __forceinline__ void scatter_item(const Args<P>& a, int64_t t) {
    int slot = a.cell_start[cell_index_of_packed(a.cell[t], a.G)] + a.rank[t];
    if (slot >= 0 && slot < a.n) a.order[slot] = (int)t;
    else atomicOr(&a.ctr->error, kErrUnstable);
}

template <class P>
__global__ void __launch_bounds__(kBlock) k_scatter(Args<P> a, int guard) {
    if (guard && !a.ctr->rebuild_flag) return;
    for (int64_t t = gtid(); t < a.n; t += (int64_t)gridDim.x * blockDim.x) scatter_item<P>(a, t);
    // counts and tile totals are no longer needed once cell_start is known
    for (int64_t t = gtid(); t < a.ncells; t += (int64_t)gridDim.x * blockDim.x) a.count[t] = 0;
    for (int64_t t = gtid(); t < a.ntiles; t += (int64_t)gridDim.x * blockDim.x) a.tile_sum[t] = 0;
}

// Makes the order inside each cell deterministic (ascending storage index).
template <class P>
__device__ __forceinline__ void cellsort_item(const Args<P>& a, int64_t c) {
    constexpr int kLocal = 8;  // cells this full are sorted in registers
    const int beg = a.cell_start[c], end = a.cell_start[c + 1];
    const int len = end - beg;
    if (len <= 1) return;
    if (len <= kLocal) {
        // all loads first (independent), then a sorting network of
        // compare-exchanges on registers, then all stores
        int k[kLocal];
#pragma unroll
        for (int u = 0; u < kLocal; u++) k[u] = u < len ? a.order[beg + u] : INT_MAX;
#pragma unroll
        for (int r = 0; r < kLocal; r++) {  // odd-even transposition sort
#pragma unroll
            for (int u = r & 1; u + 1 < kLocal; u += 2) {
                const int lo = min(k[u], k[u + 1]), hi = max(k[u], k[u + 1]);
                k[u] = lo;
                k[u + 1] = hi;
            }
        }
#pragma unroll
        for (int u = 0; u < kLocal; u++)
            if (u < len) a.order[beg + u] = k[u];
        return;
    }
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

template <class P>
__global__ void __launch_bounds__(kBlock) k_cellsort(Args<P> a, int guard) {
    if (guard && !a.ctr->rebuild_flag) return;
    int64_t c = gtid();
    if (c >= a.ncells) return;
    cellsort_item<P>(a, c);
}

// Writes the cell-ordered FP32 coordinate copy used by the neighbour search
// and, when a reorder is due, the state permuted into cell order (Sec. 3.5).
template <class P>
__device__ __forceinline__ void gather_item(const Args<P>& a, int64_t s) {
    using real = typename P::real;
    Counters* C = a.ctr;
    const int reorder = C->reorder_now;
    int i = a.order[s];
    real pbx = a.pbx[i], pby = a.pby[i], pbz = a.pbz[i];
    double ox = a.ox[i], oy = a.oy[i], oz = a.oz[i];
    real px = pair_coord(pbx, ox), py = pair_coord(pby, oy), pz = pair_coord(pbz, oz);
    a.cand[s] = make_float4(to_f32(px), to_f32(py), to_f32(pz), __int_as_float(reorder ? (int)s : i));
    if (reorder) {
        a.s_cell[s] = a.cell[i];
        a.s_perm[s] = a.perm[i];
        a.s_pbx[s] = pbx; a.s_pby[s] = pby; a.s_pbz[s] = pbz;
        a.s_ox[s] = ox; a.s_oy[s] = oy; a.s_oz[s] = oz;
        a.s_vx[s] = a.vx[i]; a.s_vy[s] = a.vy[i]; a.s_vz[s] = a.vz[i];
    }
}

template <class P>
__global__ void __launch_bounds__(kBlock) k_gather(Args<P> a, int guard) {
    using real = typename P::real;
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    int64_t s = gtid();
    if (s >= a.n) return;
    gather_item<P>(a, s);
}

// Copies the permuted state back and rewrites the current pair buffer in
// the new order (only when a reorder is due).
template <class P>
__device__ __forceinline__ void commit_item(const Args<P>& a, int64_t s) {
    Counters* C = a.ctr;
    a.cell[s] = a.s_cell[s];
    a.perm[s] = a.s_perm[s];
    auto pbx = a.s_pbx[s], pby = a.s_pby[s], pbz = a.s_pbz[s];
    double ox = a.s_ox[s], oy = a.s_oy[s], oz = a.s_oz[s];
    a.pbx[s] = pbx; a.pby[s] = pby; a.pbz[s] = pbz;
    a.ox[s] = ox; a.oy[s] = oy; a.oz[s] = oz;
    a.vx[s] = a.s_vx[s]; a.vy[s] = a.s_vy[s]; a.vz[s] = a.s_vz[s];
    typename P::pos4* pc = C->parity ? a.pB : a.pA;
    pc[s] = make_pos4(pair_coord(pbx, ox), pair_coord(pby, oy), pair_coord(pbz, oz), 0);
}

template <class P>
__global__ void __launch_bounds__(kBlock) k_commit(Args<P> a, int guard) {
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    if (!C->reorder_now) return;
    int64_t s = gtid();
    if (s >= a.n) return;
    commit_item<P>(a, s);
}

// Exact FP64 neighbour criterion r^2 < r_n^2 for atom i and atom j, whose
// cell lies at offset d from i's cell (code = (d_x+1) | (d_y+1) << 2 |
// (d_z+1) << 4), evaluated as the FP64 reference evaluates its cell pairs
// (Sec. 3.2): e = (x_i - x_j) + s L on the reported absolute coordinates,
// s = -1 / +1 when i's cell + d wraps across the upper / lower face,
// r^2 = (e_x^2 + e_y^2) + e_z^2, every operation rounded, no contraction.
// The reported coordinate k of atom i when its cell coordinate is c.
template <class P>
__device__ __noinline__ double reported_coord(const Args<P>& a, int k, int c, int i) {
    const typename P::real* pb = k == 0 ? a.pbx : (k == 1 ? a.pby : a.pbz);
    const double* o = k == 0 ? a.ox : (k == 1 ? a.oy : a.oz);
    return abs_coord(a, k, c, full_offset(pb[i], o[i]));
}

template <class P>
__device__ __noinline__ bool within_rn_fp64(const Args<P>& a, int i, int j, unsigned code) {
    int ci[3];
    unpack_cell(a.cell[i], ci[0], ci[1], ci[2]);
    double r2 = 0.0;
#pragma unroll 1
    for (int k = 0; k < 3; k++) {
        int cj = ci[k] + (int)((code >> (2 * k)) & 3u) - 1;
        double s = 0.0;
        if (cj >= a.G[k]) { cj -= a.G[k]; s = -1.0; }
        else if (cj < 0) { cj += a.G[k]; s = 1.0; }
        const double xi = reported_coord(a, k, ci[k], i);
        const double xj = reported_coord(a, k, cj, j);
        const double e = __dadd_rn(__dsub_rn(xi, xj), __dmul_rn(s, a.L[k]));
        // (e_x^2 + e_y^2) + e_z^2: the first product is added to an exact 0
        r2 = __dadd_rn(r2, __dmul_rn(e, e));
    }
    return r2 < a.rn2;
}

// Shell bin of a list entry at squared distance rr (FP32, as the build
// computes it): floor((r - r_c) kShellBins / skin), clamped to [0, 7].
template <class P>
__device__ __forceinline__ int shell_bin(const Args<P>& a, float rr) {
    const float r = rr * rsqrtf(fmaxf(rr, 1e-30f));
    const float t = (r - a.rcf) * a.shell_inv;
    return t >= 1.0f ? min((int)t, kShellBins - 1) : 0;
}

// Shell reach of a step: the smallest k in 1..kShellBins with
// r_c + k skin / kShellBins >= r_c + 2 sqrt(d2max) + margin.  A pair whose
// distance at the build was beyond that bound is farther than r_c now (each
// of its atoms has moved at most sqrt(d2max)), so only the entries below the
// k-th shell boundary need to be read.
template <class P>
__device__ __forceinline__ int shell_reach(const Args<P>& a, unsigned d2bits) {
    if (!a.shell_bins) return kShellBins;
    const float t = fmaf(2.0f, sqrtf(__uint_as_float(d2bits)), a.shell_eps) * a.shell_inv;
    return t < (float)(kShellBins - 1) ? max((int)ceilf(t), 1) : kShellBins;
}

// Neighbour-list build (Sec. 3.4): for the atom in cell-ordered slot s, scan
// the 27 cells around its cell and record every j != i with r < r_n in its
// column together with the cell-offset code.  The decision is the exact
// FP64 criterion: FP32 coordinates settle every candidate outside a narrow
// band [rn2_lo, rn2_hi) around r_n^2, the FP64 test the rest.  The three
// cells of one (c_y, c_z) row sit at base + c_x * stride in the pencil
// order, so each row costs one index computation and the six range bounds
// are read together.
//
// The scan loop only stages: every candidate with FP32 r^2 below rn2_hi is
// written, with its squared distance, to the thread's next 8-byte word
// stage[m * stride] in shared memory (a rejected candidate's word is
// overwritten by the next one), so that a candidate costs its distance, one
// store and no branch.  The loop issues kBuildUnroll candidate loads before
// it uses them (loads past a cell's end are predicated off) and loads the
// next row's cell ranges while a row runs, to hide the latency of those L1
// hits (without them the loop was latency-bound).  Afterwards the staged band
// entries get the FP64 test (rare), the survivors are written out ordered
// by shell bin (a counting sort whose bin counts sit in the bytes of one
// 64-bit word) and lim receives the number of entries below each bin
// boundary.  An atom with more than K (the stage depth) staged candidates
// is scanned again by build_all, which writes its entries in order of
// discovery with a lim of "all entries".
template <class P, bool kRows>
__device__ __noinline__ int build_all(const Args<P>& a, int64_t s) {
    const float4 ci = a.cand[s];
    const int i = __float_as_int(ci.w);
    int cx, cy, cz;
    unpack_cell(a.cell[i], cx, cy, cz);
    constexpr int cs = kRows ? 1 : 32;
    int* col = a.nbr + (kRows ? (size_t)i * (size_t)a.cap : ((size_t)(i >> 5) * (size_t)a.cap) * 32 + (i & 31));
    const int cap = a.cap, n = (int)a.n;
    int m = 0;
    for (int d = 0; d < 27; d++) {
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const int c = cell_index(wrap_add(cx, dx, a.G[0]), wrap_add(cy, dy, a.G[1]), wrap_add(cz, dz, a.G[2]), a.G);
        const int end = min(a.cell_start[c + 1], n);
        const unsigned code = (unsigned)((dx + 1) | ((dy + 1) << 2) | ((dz + 1) << 4));
        for (int t = a.cell_start[c]; t < end; t++) {
            if (t == (int)s) continue;
            const float4 pj = __ldg(a.cand + t);
            const float ex = (ci.x - (float)dx * a.wf[0]) - pj.x;
            const float ey = (ci.y - (float)dy * a.wf[1]) - pj.y;
            const float ez = (ci.z - (float)dz * a.wf[2]) - pj.z;
            const float rr = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            if (!(rr < a.rn2_hi)) continue;
            const int j = __float_as_int(pj.w);
            if (!(rr < a.rn2_lo) && !within_rn_fp64(a, i, j, code)) continue;
            if (m < cap) col[(size_t)m * cs] = j | (int)(code << kCodeShift);
            m++;
        }
    }
    return m;
}

// The direct build's second pass, run only for an atom that met a
// candidate in the band: the band candidates (same FP32 distance as the
// first pass), decided by the exact FP64 criterion and appended after the m
// entries already written.  Returns the new count.
template <class P, bool kRows>
__device__ __noinline__ int build_band(const Args<P>& a, int64_t s, int m) {
    const float4 ci = a.cand[s];
    const int i = __float_as_int(ci.w);
    int cx, cy, cz;
    unpack_cell(a.cell[i], cx, cy, cz);
    constexpr int cs = kRows ? 1 : 32;
    int* col = a.nbr + (kRows ? (size_t)i * (size_t)a.cap : ((size_t)(i >> 5) * (size_t)a.cap) * 32 + (i & 31));
    const int cap = a.cap, n = (int)a.n;
    for (int d = 0; d < 27; d++) {
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const int c = cell_index(wrap_add(cx, dx, a.G[0]), wrap_add(cy, dy, a.G[1]), wrap_add(cz, dz, a.G[2]), a.G);
        const int end = min(a.cell_start[c + 1], n);
        const unsigned code = (unsigned)((dx + 1) | ((dy + 1) << 2) | ((dz + 1) << 4));
        for (int t = a.cell_start[c]; t < end; t++) {
            const float4 pj = __ldg(a.cand + t);
            const float ex = (ci.x - (float)dx * a.wf[0]) - pj.x;
            const float ey = (ci.y - (float)dy * a.wf[1]) - pj.y;
            const float ez = (ci.z - (float)dz * a.wf[2]) - pj.z;
            const float rr = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            if (!(rr >= a.rn2_lo && rr < a.rn2_hi) || t == (int)s) continue;
            const int j = __float_as_int(pj.w);
            if (!within_rn_fp64(a, i, j, code)) continue;
            if (m < cap) col[(size_t)m * cs] = j | (int)(code << kCodeShift);
            m++;
        }
    }
    return m;
}

// kDirect: the direct form for lists longer than the stage (dense or long-
// range workloads): each accepted entry goes straight to the list, in order
// of discovery, with a lim of "all entries"; a candidate in the band only
// marks the atom, and build_band decides the marked atom's band candidates
// afterwards (the rare FP64 path then costs the scan loop no registers).
template <class P, bool kSort, bool kRows, int K, bool kDirect = false>
__device__ __forceinline__ int build_item_t(const Args<P>& a, int64_t s, int2* stage, int stride) {
    Counters* C = a.ctr;
    int m = 0;  // staged candidates (FP32 r^2 < rn2_hi)
    const float4 ci = a.cand[s];
    const int i = __float_as_int(ci.w);
    int cx, cy, cz;
    unpack_cell(a.cell[i], cx, cy, cz);
    constexpr int cs = kRows ? 1 : 32;
    int* col = a.nbr + (kRows ? (size_t)i * (size_t)a.cap : ((size_t)(i >> 5) * (size_t)a.cap) * 32 + (i & 31));
    const int cap = a.cap, n = (int)a.n, self = (int)s;
    const float hi2 = a.rn2_hi, lo2d = a.rn2_lo;
    bool unsure = false;  // (direct form) a candidate in the band was met
    const int xs[3] = {wrap_add(cx, -1, a.G[0]), cx, wrap_add(cx, 1, a.G[0])};
    const float qxs[3] = {ci.x + a.wf[0], ci.x, ci.x - a.wf[0]};  // x seen from cells x-1, x, x+1
    // candidate ranges of the three cells of row r = (d_y + 1) + 3 (d_z + 1)
    auto row_bounds = [&](int r, int lo[3], int hi[3]) {
        const int y = wrap_add(cy, r % 3 - 1, a.G[1]), z = wrap_add(cz, r / 3 - 1, a.G[2]);
        const PencilRow pr = pencil_row(y, z, a.G);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int c = pr.base + xs[k] * pr.stride;
            lo[k] = a.cell_start[c];
            hi[k] = min(a.cell_start[c + 1], n);
        }
    };
    int lo[3], hi[3];
    row_bounds(0, lo, hi);
#pragma unroll 1
    for (int r = 0; r < 9; r++) {
        int nlo[3], nhi[3];  // the next row's bounds, loaded while this row runs
        if (kBuildPrefetch) row_bounds(r < 8 ? r + 1 : r, nlo, nhi);
        const int dy = r % 3 - 1, dz = r / 3 - 1;
        const float qz = ci.z - (float)dz * a.wf[2];
        const float qy = ci.y - (float)dy * a.wf[1];
        const unsigned code_yz = ((unsigned)(dy + 1) << 2) | ((unsigned)(dz + 1) << 4);
        auto stage_one = [&](const float4& pj, float qx, int code, int t) {
            const float ex = qx - pj.x;
            const float ey = qy - pj.y;
            const float ez = qz - pj.z;
            const float rr = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            if constexpr (kDirect) {
                const bool take = rr < lo2d && t != self;
                unsure |= !(rr < lo2d) && rr < hi2;
                if (take && m < cap) col[(size_t)m * cs] = __float_as_int(pj.w) | code;
                m += take ? 1 : 0;
            } else {
                if (m < K) stage[m * stride] = make_int2(__float_as_int(pj.w) | code, __float_as_int(rr));
                m += (rr < hi2 && t != self) ? 1 : 0;
            }
        };
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float qx = qxs[k];
            const int code = (int)(((unsigned)k | code_yz) << kCodeShift);
            const int end = hi[k];
            for (int t = lo[k]; t < end; t += kBuildUnroll) {
                float4 pj[kBuildUnroll];  // all loads first
#pragma unroll
                for (int u = 0; u < kBuildUnroll; u++)
                    pj[u] = (u == 0 || t + u < end) ? __ldg(a.cand + t + u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < kBuildUnroll; u++)
                    if (u == 0 || t + u < end) stage_one(pj[u], qx, code, t + u);
            }
        }
        if (kBuildPrefetch) {
#pragma unroll
            for (int k = 0; k < 3; k++) { lo[k] = nlo[k]; hi[k] = nhi[k]; }
        } else if (r < 8) {
            row_bounds(r + 1, lo, hi);
        }
    }
    if constexpr (kDirect) {
        if (unsure) m = build_band<P, kRows>(a, s, m);
        a.nn[i] = m < cap ? m : cap;
        if constexpr (kSort) {
#pragma unroll
            for (int k = 1; k < kShellBins; k++) a.lim[(size_t)(k - 1) * a.n + i] = 255;
        }
    } else if (m > K) {  // rare: too long for the stage
        m = build_all<P, kRows>(a, s);
        const int kept = m < cap ? m : cap;
        a.nn[i] = kept;
        if constexpr (kSort) {
#pragma unroll
            for (int k = 1; k < kShellBins; k++) a.lim[(size_t)(k - 1) * a.n + i] = 255;
        }
    } else {
        // FP64 test of the band entries; bin of each survivor (kShellBins
        // marks a rejected one) and the bin counts in the bytes of (hhi:hlo)
        const float lo2 = a.rn2_lo;
        unsigned hlo = 0u, hhi = 0u;
        int kept = 0;
        for (int t = 0; t < m; t++) {
            const int2 e = stage[t * stride];
            const float rr = __int_as_float(e.y);
            bool keep = true;
            if (!(rr < lo2)) keep = within_rn_fp64(a, i, e.x & kIndexMask, (unsigned)e.x >> kCodeShift);
            const int b = !keep ? kShellBins : (kSort ? shell_bin(a, rr) : 0);
            stage[t * stride].y = b;
            kept += keep ? 1 : 0;
            const unsigned inc = keep ? 1u << (8 * (b & 3)) : 0u;
            hlo += b < 4 ? inc : 0u;
            hhi += b < 4 ? 0u : inc;
        }
        // byte b of incl: entries of bins 0..b, i.e. those below the
        // boundary r_c + (b + 1) skin / kShellBins (no byte exceeds K)
        const unsigned long long incl = (((unsigned long long)hhi << 32) | hlo) * 0x0101010101010101ull;
        const unsigned long long first = incl << 8;  // exclusive: first slot of each bin
        unsigned nlo = (unsigned)first, nhi = (unsigned)(first >> 32);
        for (int t = 0; t < m; t++) {
            const int2 e = stage[t * stride];
            const int b = e.y;
            if (b == kShellBins) continue;
            const int sh = 8 * (b & 3);
            const int dst = (int)(((b < 4 ? nlo : nhi) >> sh) & 0xffu);
            const unsigned inc = 1u << sh;
            nlo += b < 4 ? inc : 0u;
            nhi += b < 4 ? 0u : inc;
            if (dst < cap) col[(size_t)dst * cs] = e.x;
        }
        a.nn[i] = kept < cap ? kept : cap;
        if constexpr (kSort) {
#pragma unroll
            for (int k = 1; k < kShellBins; k++)
                a.lim[(size_t)(k - 1) * a.n + i] = (unsigned char)(incl >> (8 * (k - 1)));
        }
        m = kept;
    }
    if (m > cap) {
        atomicOr(&C->error, kErrOverflow);
        atomicMax(&C->need_cap, m);
    }
    return m;
}

// K: the stage depth (8-byte words per thread at stage[t * stride]).
template <class P, bool kRows = false, int K = kBuildStage, bool kDirect = false>
__device__ __forceinline__ int build_item(const Args<P>& a, int64_t s, int2* stage, int stride) {
    return a.shell_bins ? build_item_t<P, true, kRows, K, kDirect>(a, s, stage, stride)
                        : build_item_t<P, false, kRows, K, kDirect>(a, s, stage, stride);
}

template <class P, bool kRows = false, bool kDirect = false>
__global__ void __launch_bounds__(kBuildBlock, 8) k_build(Args<P> a, int guard) {
    constexpr int kWarps = kBuildBlock / 32;
    __shared__ int s_max[kWarps], s_sum[kWarps];
    __shared__ int2 s_stage[kDirect ? 1 : kBuildStage * kBuildBlock];
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    const int64_t s = gtid();
    const int m = s < a.n ? build_item<P, kRows, kBuildStage, kDirect>(a, s, s_stage + threadIdx.x, kBuildBlock) : 0;
    // block maximum and sum of the list lengths (m <= 512, so the block's
    // sum fits an int)
    int bm = m, bs = m;
    for (int o = 16; o > 0; o >>= 1) {
        bm = max(bm, __shfl_xor_sync(0xffffffffu, bm, o));
        bs += __shfl_xor_sync(0xffffffffu, bs, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_max[threadIdx.x >> 5] = bm;
        s_sum[threadIdx.x >> 5] = bs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kWarps; w++) {
            bm = max(bm, s_max[w]);
            bs += s_sum[w];
        }
        atomicMax(&C->max_nn, bm);
        atomicAdd((unsigned long long*)&C->list_entries, (unsigned long long)bs);
    }
}

// ---------------------------------------------------------------------------
// Warp-cooperative neighbour-list build (Sec. 3.4, W_{m,i} and m_i)
// ---------------------------------------------------------------------------
//
// One thread block per x slice of a pencil (the up to 4 x 4 cells of one
// tile at one c_x, consecutive in the cell order) and one warp per cell of
// the slice.  The warp gathers the candidates of the 27 cells around its
// home cell into shared memory once -- each shifted into the home cell's
// frame (x_j + d w) and tagged with its entry j | code << kCodeShift -- and
// then takes the home atoms one at a time: every lane tests one candidate,
// so the warp has no per-lane loops of uneven length and every candidate is
// loaded once per home cell instead of once per home atom.  The decision is
// the one of the thread-per-atom build (FP32 outside a narrow band around
// r_n^2, the exact FP64 criterion inside it).  Accepted entries are
// compacted by ballot into a per-warp stage; a list of at most kWcSort
// entries is then written ordered by shell bin, each lane placing one entry
// at (entries of lower bins) + (entries of its bin before it), both counted
// from three ballots over the bits of the bin, and lim receives the counts
// below each bin boundary.  A longer list keeps its order of discovery and a
// lim of "all entries".
constexpr int kWcBatch = 192;   // candidates staged per warp at a time
constexpr int kWcSort = 32;     // lists up to this long are sorted by shell bin
constexpr int kWcWarps = kWcThreads / 32;  // one per cell of a slice

struct WcWarp {
    float4 cand[kWcBatch];
    int2 stage[kWcSort];
};

// Cell-offset code (d_x+1) | (d_y+1) << 2 | (d_z+1) << 4 of stencil cell
// c = (d_x+1) + 3 (d_y+1) + 9 (d_z+1).
__device__ __forceinline__ unsigned c9_code(int c) {
    const unsigned x = (unsigned)(c % 3), y = (unsigned)((c / 3) % 3), z = (unsigned)(c / 9);
    return x | (y << 2) | (z << 4);
}

// Lanes (of the valid mask V, bins b held as the bit masks M0, M1, M2) whose
// bin is below t.
__device__ __forceinline__ unsigned bins_below(int t, unsigned V, unsigned M0, unsigned M1, unsigned M2) {
    const unsigned E2 = (t & 4) ? M2 : ~M2, E1 = (t & 2) ? M1 : ~M1;
    const unsigned lt2 = (t & 4) ? (V & ~M2) : 0u;
    const unsigned lt1 = (t & 2) ? (V & E2 & ~M1) : 0u;
    const unsigned lt0 = (t & 1) ? (V & E2 & E1 & ~M0) : 0u;
    return lt2 | lt1 | lt0;
}

template <class P>
__global__ void __launch_bounds__(kWcThreads, 2) k_build_wc(Args<P> a, int guard) {
    __shared__ WcWarp s_wc[kWcWarps];
    __shared__ int s_max[kWcWarps];
    __shared__ long long s_sum[kWcWarps];
    Counters* C = a.ctr;
    if (guard && !C->rebuild_flag) return;
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    WcWarp& W = s_wc[wid];
    const int n = (int)a.n, cap = a.cap, cs = list_stride(a);
    const float lo2 = a.rn2_lo, hi2 = a.rn2_hi;
    // the slice of this block and the home cell of this warp
    const int nty = (a.G[1] + 3) / 4;
    const int cx = (int)(blockIdx.x % (unsigned)a.G[0]);
    const int tile = (int)(blockIdx.x / (unsigned)a.G[0]);
    const int y0 = (tile % nty) * 4, z0 = (tile / nty) * 4;
    const int hy = min(4, a.G[1] - y0), hz = min(4, a.G[2] - z0);
    int mx = 0;
    long long sum = 0;
    if (wid < hy * hz) {
        const int cy = y0 + wid % hy, cz = z0 + wid / hy;
        // this lane's stencil cell (lanes 0..26), d = (dx, dy, dz)
        const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
        int start = 0, cnt = 0;
        if (lane < 27) {
            const int c2 = cell_index(wrap_add(cx, dx, a.G[0]), wrap_add(cy, dy, a.G[1]), wrap_add(cz, dz, a.G[2]), a.G);
            start = a.cell_start[c2];
            cnt = max(min(a.cell_start[c2 + 1], n) - start, 0);
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int excl = incl - cnt;
        const int K = __shfl_sync(kFull, incl, 31);
        const int nh = __shfl_sync(kFull, cnt, 13);  // lane 13: the home cell itself
        const int h0 = __shfl_sync(kFull, excl, 13);
        const int hs = __shfl_sync(kFull, start, 13);
        for (int h = 0; h < nh; h++) {
            // the home atoms are the staged candidates of lane 13's cell (no
            // shift) as long as they lie in the first batch
            const bool staged_home = h0 + h < kWcBatch;
            float4 qi;
            if (!staged_home) qi = a.cand[hs + h];
            const int kself = h0 + h;
            int m = 0;
            int i = -1;
            int* col = nullptr;
            for (int b0 = 0; b0 < K; b0 += kWcBatch) {
                if (h == 0 || K > kWcBatch) {  // (re)fill the staged candidates
                    // lanes over candidates: candidate k lies in the stencil
                    // cell c = number of cells whose inclusive count is <= k
                    // (binary search over the scan), slot start_c + k - excl_c
                    __syncwarp();
                    const int kend = min(K - b0, kWcBatch);
#pragma unroll 2
                    for (int r = 0; r < kend; r += 32) {
                        const int kl = r + lane, k = b0 + kl;
                        int c = 0;
#pragma unroll
                        for (int st = 16; st > 0; st >>= 1)
                            if (__shfl_sync(kFull, incl, c + st - 1) <= k) c += st;
                        const int sc = __shfl_sync(kFull, start, c), ec = __shfl_sync(kFull, excl, c);
                        if (kl < kend) {
                            const int ddx = c % 3 - 1, ddy = (c / 3) % 3 - 1, ddz = c / 9 - 1;
                            const float4 pj = __ldg(a.cand + sc + (k - ec));
                            W.cand[kl] = make_float4(
                                fmaf((float)ddx, a.wf[0], pj.x), fmaf((float)ddy, a.wf[1], pj.y),
                                fmaf((float)ddz, a.wf[2], pj.z),
                                __int_as_float(__float_as_int(pj.w) | (int)((unsigned)c9_code(c) << kCodeShift)));
                        }
                    }
                    __syncwarp();
                }
                if (b0 == 0) {
                    if (staged_home) qi = W.cand[kself];
                    i = __float_as_int(qi.w) & kIndexMask;
                    col = a.nbr + list_base(a, i);
                }
                const int kend = min(K - b0, kWcBatch);
                for (int r = 0; r < kend; r += 32) {
                    const int kl = r + lane;
                    bool take = false, unsure = false;
                    int e = 0;
                    float rr = 0.0f;
                    if (kl < kend && b0 + kl != kself) {
                        const float4 c = W.cand[kl];
                        const float ex = qi.x - c.x, ey = qi.y - c.y, ez = qi.z - c.z;
                        rr = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                        e = __float_as_int(c.w);
                        take = rr < lo2;
                        unsure = !take && rr < hi2;
                    }
                    if (unsure) take = within_rn_fp64(a, i, e & kIndexMask, (unsigned)e >> kCodeShift);
                    const unsigned bal = __ballot_sync(kFull, take);
                    const int dst = m + __popc(bal & lt);
                    if (take) {
                        if (dst < kWcSort) W.stage[dst] = make_int2(e, __float_as_int(rr));
                        else if (dst < cap) col[(size_t)dst * cs] = e;
                    }
                    m += __popc(bal);
                }
            }
            __syncwarp();
            if (lane == 0) a.nn[i] = min(m, cap);
            if (a.shell_bins && m <= kWcSort && m <= cap) {
                const bool v = lane < m;
                int b = 0, e = 0;
                if (v) {
                    const int2 st = W.stage[lane];
                    e = st.x;
                    b = shell_bin(a, __int_as_float(st.y));
                }
                const unsigned V = __ballot_sync(kFull, v);
                const unsigned M0 = __ballot_sync(kFull, (b & 1) != 0), M1 = __ballot_sync(kFull, (b & 2) != 0),
                               M2 = __ballot_sync(kFull, (b & 4) != 0);
                if (v) {
                    const unsigned same = V & ((b & 4) ? M2 : ~M2) & ((b & 2) ? M1 : ~M1) & ((b & 1) ? M0 : ~M0);
                    col[(size_t)(__popc(bins_below(b, V, M0, M1, M2)) + __popc(same & lt)) * cs] = e;
                }
                if (lane >= 1 && lane < kShellBins)
                    a.lim[(size_t)(lane - 1) * a.n + i] = (unsigned char)__popc(bins_below(lane, V, M0, M1, M2));
            } else {
                const int ns = min(min(m, kWcSort), cap);
                if (lane < ns) col[(size_t)lane * cs] = W.stage[lane].x;
                if (a.shell_bins && lane >= 1 && lane < kShellBins) a.lim[(size_t)(lane - 1) * a.n + i] = 0xff;
            }
            if (m > cap && lane == 0) {
                atomicOr(&C->error, kErrOverflow);
                atomicMax(&C->need_cap, m);
            }
            mx = max(mx, m);
            sum += m;
            __syncwarp();  // the stage is reused by the next home atom
        }
    }
    if (lane == 0) {
        s_max[wid] = mx;
        s_sum[wid] = sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int bm = 0;
        long long bs = 0;
        for (int w = 0; w < kWcWarps; w++) {
            bm = max(bm, s_max[w]);
            bs += s_sum[w];
        }
        atomicMax(&C->max_nn, bm);
        atomicAdd((unsigned long long*)&C->list_entries, (unsigned long long)bs);
    }
}

// Closes a rebuild: counters, reorder bookkeeping, flag cleared, and the
// running maximum of the displacement restarted.  One warp.
template <class P>
__global__ void k_rebuild_done(Args<P> a, int guard) {
    Counters* C = a.ctr;
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const bool run = !guard || C->rebuild_flag;
    __syncwarp();  // every lane has read the flag before lane 0 clears it
    if (!run) return;
    if (a.d2b)
        for (int b = threadIdx.x; b < kD2Buckets; b += 32) a.d2b[b * 32] = 0u;
    if (threadIdx.x != 0) return;
    C->rebuilds += 1;
    if (C->reorder_now) {
        C->reorders += 1;
        C->since_reorder = 0;
        C->reorder_now = 0;
    }
    C->rebuild_flag = 0;
    C->d2max = 0u;  // displacements now count from the new build
    C->reach = shell_reach(a, 0u);
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
// reorder_interval steps have passed (Sec. 5.5).
__device__ __forceinline__ int decide_rebuild(Counters* C, int cell_list_only, int interval) {
    int need = (C->far_flag != 0u) || cell_list_only;
    C->far_flag = 0u;
    C->rebuild_flag = need;
    C->reorder_now = need && interval > 0 && C->since_reorder >= interval;
    return need;
}

// Half kick in the velocity precision.
__device__ __forceinline__ float kick(const Args<Mixed>& a, float v, float f) { return fmaf(a.hf, f, v); }
__device__ __forceinline__ double kick(const Args<F64>& a, double v, double f) { return fma(a.h, f, v); }

// This block's word of the running maximum of the squared displacement.
template <class P>
__device__ __forceinline__ unsigned* d2_word(const Args<P>& a) {
    return a.d2b ? a.d2b + (blockIdx.x % kD2Buckets) * 32 : &a.ctr->d2max;
}

// The running maximum over all words (warp-wide: every lane of the warp
// must call it and gets the result).  Reads past L1.
template <class P>
__device__ __forceinline__ unsigned d2_gather_warp(const Args<P>& a) {
    unsigned v = 0u;
    if (a.d2b) {
        for (int b = threadIdx.x & 31; b < kD2Buckets; b += 32) v = max(v, __ldcg(a.d2b + b * 32));
    } else {
        v = __ldcg(&a.ctr->d2max);
    }
    return __reduce_max_sync(0xffffffffu, v);
}

// Bits of a squared displacement as FP32 (>= 0, so the unsigned order of
// the bits is the order of the values).
__device__ __forceinline__ unsigned d2_bits(float d2) { return __float_as_uint(d2); }
__device__ __forceinline__ unsigned d2_bits(double d2) { return __float_as_uint(cvt::f32(d2)); }

// Largest value over the warp, merged by lane 0 into the running maximum
// *dst.  The atomic is skipped when a value *dst already held is not
// smaller: *dst only grows while a kernel runs (it is cleared in another
// kernel), so the read may come from L1 and be stale, and the atomics,
// which all go to one address, stay few.  kL2: read past L1 (a persistent
// kernel whose team clears *dst between steps).  Every lane of the warp
// must call it.
template <bool kL2 = false>
__device__ __forceinline__ void warp_max_into(unsigned v, unsigned* dst) {
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && v > (kL2 ? __ldcg(dst) : *dst)) atomicMax(dst, v);
}

// One atom of k_kickdrift; returns whether it has moved skin/2 and sets
// d2b to the bits of its squared displacement.
template <class P>
__device__ __forceinline__ bool kickdrift_item(const Args<P>& a, int64_t i, typename P::pos4* pc, unsigned& d2b) {
    using real = typename P::real;
    using vel = typename P::vel;
    vel vx = kick(a, a.vx[i], a.fx[i]);
    vel vy = kick(a, a.vy[i], a.fy[i]);
    vel vz = kick(a, a.vz[i], a.fz[i]);
    double ox = drift(a.ox[i], vx, a.dt);
    double oy = drift(a.oy[i], vy, a.dt);
    double oz = drift(a.oz[i], vz, a.dt);
    real px, py, pz;
    real d2 = moved(a.pbx[i], ox, px) + moved(a.pby[i], oy, py) + moved(a.pbz[i], oz, pz);
    a.vx[i] = vx; a.vy[i] = vy; a.vz[i] = vz;
    a.ox[i] = ox; a.oy[i] = oy; a.oz[i] = oz;
    pc[i] = make_pos4(px, py, pz, 0);
    d2b = d2_bits(d2);
    if constexpr (P::kFp64) return d2 >= a.thr2;
    else return d2 >= a.thr2f;
}

// First half of the first step of an md_step call (Sec. 3.1 (a)): half kick
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
    unsigned d2b = 0u;
    if (!err && i < a.n) far = kickdrift_item<P>(a, i, par ? a.pB : a.pA, d2b);
    if (__any_sync(0xffffffffu, far) && (threadIdx.x & 31) == 0) atomicOr(&C->far_flag, 1u);
    warp_max_into(d2b, d2_word(a));
    if (last_block_done(C)) {
        const unsigned d2 = threadIdx.x < 32 ? d2_gather_warp(a) : 0u;
        if (threadIdx.x == 0) {
            if (!err) {
                C->steps_left = nsteps;
                decide_rebuild(C, a.cell_list_only, a.reorder_interval);
                C->d2max = d2;
                C->reach = shell_reach(a, d2);
            }
            C->ticket = 0;
        }
    }
}

// Entries of atom i < n to read at shell reach k (all of them outside
// 1..kShellBins-1, where no plane applies).
template <class P>
__device__ __forceinline__ int list_count(const Args<P>& a, int64_t i, int k) {
    int c = 0xff;
    if (k >= 1 && k < kShellBins) c = a.lim[(size_t)(k - 1) * a.n + i];
    return c != 0xff ? c : a.nn[i];
}

// Stages the first rows of the warp's neighbour column block in shared
// memory (rows below the capacity always exist; unused ones are ignored)
// and reads the number of entries of atom i that the step's shell reach
// (from the counters) leaves to read.  Every lane of the warp must call it.
template <class P, bool kCells, bool kRows = false>
__device__ __forceinline__ void stage_rows(const Args<P>& a, int64_t i, int reach, int* rows, int& cnt,
                                           int& staged, const int*& col) {
    cnt = 0;
    staged = 0;
    col = nullptr;
    if constexpr (!kCells) {
        if (!kRows && (i & ~(int64_t)31) < a.n) {  // the warp's column block exists
            staged = min(a.cap, kStageRows);
            const int* blk = a.nbr + (size_t)(i >> 5) * (size_t)a.cap * 32;
            for (int c = threadIdx.x & 31; c < staged * 8; c += 32) cp_async16(rows + 4 * c, blk + 4 * c);
        }
        if (i < a.n) {
            cnt = list_count(a, i, reach);
            col = a.nbr + (kRows ? (size_t)i * (size_t)a.cap : ((size_t)(i >> 5) * (size_t)a.cap) * 32 + (i & 31));
        }
    }
}
template <bool kCells>
__device__ __forceinline__ void stage_wait() {
    if constexpr (!kCells) {  // every lane that issued copies waits for them
        cp_async_wait_all();
        __syncwarp();
    }
}

// The per-atom part of a step (Sec. 3.1 (c)-(e) and (a) of the next step):
// forces of atom i, then either the final-step work (v_n, stored forces,
// KE/PE/W terms) or the next half kick, the drift into the other pair
// buffer and the skin/2 test.  Shared by the grid kernel and the
// per-replica engine.
template <class P, bool kCells, bool kFinal, bool kLdg = true, bool kRows = false, bool kHwCvt = false>
__device__ __forceinline__ void step_atom(const Args<P>& a, int64_t i, bool in, bool active, bool init, bool energy,
                                          int cnt, const int* col, const int* rows, int staged,
                                          const typename P::pos4* __restrict__ pc, typename P::pos4* pn,
                                          const typename P::pos4* s_shift, typename Queue<P>::item* s_queue,
                                          bool& far, bool& close, double& ke, double& pe, double& vir,
                                          unsigned& d2b) {
    using real = typename P::real;
    using vel = typename P::vel;
    using pos4 = typename P::pos4;
    if (!(active && in)) return;
    {
        const pos4 qi = ld_pos4(pc + i);
        const real qx = qi.x, qy = qi.y, qz = qi.z;
        typename AccOf<P>::type acc;
        if (kFinal && energy) {
            if constexpr (kCells) forces_from_cells<P, kFinal>(a, (int)i, qx, qy, qz, pc, acc);
            else if constexpr (P::kFp64)
                forces_from_list<P, kFinal>(a, cnt, col, rows, staged, qx, qy, qz, pc, s_shift, s_queue, acc);
            else forces_mixed<kFinal, kLdg, kRows>(a, cnt, col, rows, staged, qx, qy, qz, pc, acc);
        } else {
            if constexpr (kCells) forces_from_cells<P, false>(a, (int)i, qx, qy, qz, pc, acc);
            else if constexpr (P::kFp64)
                forces_from_list<P, false>(a, cnt, col, rows, staged, qx, qy, qz, pc, s_shift, s_queue, acc);
            else forces_mixed<false, kLdg, kRows>(a, cnt, col, rows, staged, qx, qy, qz, pc, acc);
        }
        close = acc.close != 0;
        real fx = acc.force_x(), fy = acc.force_y(), fz = acc.force_z();
        vel vx = a.vx[i], vy = a.vy[i], vz = a.vz[i];
        const real pbx = a.pbx[i], pby = a.pby[i], pbz = a.pbz[i];
        double ox = a.ox[i], oy = a.oy[i], oz = a.oz[i];
        if (!init) {
            vx = kick(a, vx, fx);
            vy = kick(a, vy, fy);
            vz = kick(a, vz, fz);
        }
        if (energy) {
            a.fx[i] = fx; a.fy[i] = fy; a.fz[i] = fz;
            double dvx, dvy, dvz;
            if constexpr (P::kFp64) { dvx = vx; dvy = vy; dvz = vz; }
            else { dvx = cvt::f64(vx); dvy = cvt::f64(vy); dvz = cvt::f64(vz); }
            ke = 0.5 * (dvx * dvx + dvy * dvy + dvz * dvz);
            pe = 0.5 * acc.energy();
            vir = 0.5 * acc.virial();
            if (!init) { a.vx[i] = vx; a.vy[i] = vy; a.vz[i] = vz; }
        } else {
            vx = kick(a, vx, fx);
            vy = kick(a, vy, fy);
            vz = kick(a, vz, fz);
            ox = drift(ox, vx, a.dt);
            oy = drift(oy, vy, a.dt);
            oz = drift(oz, vz, a.dt);
            real px, py, pz;
            real d2 = moved<kHwCvt>(pbx, ox, px) + moved<kHwCvt>(pby, oy, py) + moved<kHwCvt>(pbz, oz, pz);
            a.vx[i] = vx; a.vy[i] = vy; a.vz[i] = vz;
            a.ox[i] = ox; a.oy[i] = oy; a.oz[i] = oz;
            pn[i] = make_pos4(px, py, pz, 0);
            d2b = d2_bits(d2);
            if constexpr (P::kFp64) far = d2 >= a.thr2;
            else far = d2 >= a.thr2f;
        }
    }
}

// The counters a step's closing work reads, loaded by lane 0 in one round
// trip to L2 (other blocks of the step wrote the flags: read past L1).
struct CloseIn {
    int err = 0, par = 0, close = 0, pend = 0;
    unsigned far = 0u;
    long long left = 0, step = 0, since = 0;
};
__device__ __forceinline__ CloseIn read_close_in(const Counters* C) {
    CloseIn r;
    if ((threadIdx.x & 31) == 0) {
        r.err = __ldcg(&C->error);
        r.par = __ldcg(&C->parity);
        r.close = __ldcg(&C->close_flag);
        r.far = __ldcg(&C->far_flag);
        r.left = __ldcg(&C->steps_left);
        r.step = __ldcg(&C->step);
        r.since = __ldcg(&C->since_reorder);
        r.pend = __ldcg(&C->rebuild_flag);
    }
    return r;
}

template <class P>
__device__ __forceinline__ void close_step(const Args<P>& a, const CloseIn& in, unsigned d2, int err, long long left,
                                           int par, bool init, bool last, bool misplaced, bool active,
                                           cudaGraphConditionalHandle next, int has_next);

// Force + integration kernel (Sec. 3.1 (c)-(e) of one step and (a) of the
// next).  A full step: forces f_n, v_n = v_{n-1/2} + f_n dt/2,
// v_{n+1/2} = v_n + f_n dt/2, o += v_{n+1/2} dt into the other pair buffer
// and the skin/2 test.  The kFinal variant also handles the last step of an
// md_step call (forces, v_n, PE/W/KE partials, no drift) and mode
// kModeInit (forces of a freshly loaded state); the plain variant, used for
// every other step, carries no energy accumulators.  The closing work
// (counters, the rebuild decision, in a graph the next conditional rebuild)
// runs in k_step_tail, or with kStepTailNode off in the last block.  A step
// whose rebuild is due and has not run (a graph checks every
// kRebuildEvery steps) does nothing.
//
// The template arguments after kFinal select the kernel variants of the
// paper's ablations (mixed list form): kB threads per block (Table 6),
// gathers through plain coherent loads instead of the read-only path
// (kLdg = false; the texture cache of Sec. 4.4), and the list stored with
// each atom's entries contiguous (kRows; W transposed, no row staging).  A
// variant with kB != kBlock serves the plain steps only: the final step,
// which writes per-block energy partials, always runs with kBlock.
template <class P, bool kCells, bool kFinal, int kB = kBlock, bool kLdg = true, bool kRows = false>
__global__ void __launch_bounds__(kB, P::kFp64 ? 3 : 5 * kBlock / kB) k_step(Args<P> a, int mode,
                                                                             cudaGraphConditionalHandle next,
                                                                             int has_next) {
    static_assert(!kFinal || kB == kBlock, "the final step runs with kBlock threads");
    using real = typename P::real;
    using vel = typename P::vel;
    using pos4 = typename P::pos4;
    __shared__ double shs[kB / 32];
    constexpr bool kTable = P::kFp64 && !kCells;  // shift table and pair queue (FP64 list form)
    __shared__ pos4 s_shift[kTable ? 64 : 1];
    __shared__ typename Queue<P>::item s_queue[kTable ? Queue<P>::kSlots * kB : 1];
    __shared__ __align__(16) int s_rows[(kCells || kRows) ? 4 : kStageRows * kB];
    Counters* C = a.ctr;
    if constexpr (kTable) fill_shift_table<P>(a, s_shift);
    // Requests that do not depend on the counters go out first, so their
    // latency overlaps the counter read: the first rows of the warp's
    // neighbour column block (copied to shared memory; rows below the
    // capacity always exist, unused ones are ignored) and the number of
    // entries to read.  The pair coordinate q_i comes from the current pair
    // buffer (bit-identical to pb + o rounded, which wrote it); pb and o are
    // read after the force loop, where they are needed.
    const int64_t i = gtid();
    const bool in = i < a.n;
    int cnt, staged;
    const int* col;
    int* rows = s_rows + (threadIdx.x >> 5) * (kStageRows * 32);
    stage_rows<P, kCells, kRows>(a, i, C->reach, rows, cnt, staged, col);
    stage_wait<kCells || kRows>();
    // the FP64 list form's block barrier also orders the table fill before its use
    const View vw = (kTable || !kStepTailNode || !kWarpView) ? load_view(C) : load_view_warp(C);
    const int err = vw.err;
    const long long left = vw.left;
    const int par = vw.par;
    const bool init = kFinal && (mode == kModeInit);
    const bool last = kFinal && !init && left == 1;
    const bool misplaced = !kFinal && left == 1;  // a plain node must never run a call's last step
    // a step whose rebuild is due but has not run (a graph checks for
    // rebuilds every kRebuildEvery steps) waits: it does nothing, and the
    // call runs one step more at its end
    const bool active = init || (err == 0 && left > 0 && !misplaced && !vw.pend);
    const bool energy = init || last;
    const pos4* pc = par ? a.pB : a.pA;
    pos4* pn = par ? a.pA : a.pB;
    bool far = false, close = false;
    double ke = 0.0, pe = 0.0, vir = 0.0;
    unsigned d2b = 0u;
    step_atom<P, kCells, kFinal, kLdg, kRows, true>(a, i, in, active, init, energy, cnt, col, rows, staged, pc, pn,
                                                    s_shift, s_queue, far, close, ke, pe, vir, d2b);
    if (__any_sync(0xffffffffu, far) && (threadIdx.x & 31) == 0) atomicOr(&C->far_flag, 1u);
    if (__any_sync(0xffffffffu, close) && (threadIdx.x & 31) == 0) atomicOr(&C->close_flag, 1);
    warp_max_into(d2b, d2_word(a));  // the running maximum of the squared displacement
    if constexpr (kFinal) {
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
    }
    if constexpr (!kStepTailNode) {
        if (last_block_done(C) && threadIdx.x < 32) {
            const CloseIn in = read_close_in(C);
            const unsigned d2 = d2_gather_warp(a);
            close_step<P>(a, in, d2, err, left, par, init, last, misplaced, active, next, has_next);
        }
    }
}

// The step's closing work (Sec. 3.1 (b) for the next step): error bits,
// counters, the rebuild decision and the shell reach, and in a graph the
// next conditional rebuild node.  Lane 0 of one warp does it after all of
// the step's blocks have finished, from the counters in `in` (read_close_in)
// and the step's largest squared displacement d2 (d2_gather_warp).
template <class P>
__device__ __forceinline__ void close_step(const Args<P>& a, const CloseIn& in, unsigned d2, int err, long long left,
                                           int par, bool init, bool last, bool misplaced, bool active,
                                           cudaGraphConditionalHandle next, int has_next) {
    Counters* C = a.ctr;
    const int err0 = in.err, close0 = in.close;
    const unsigned far0 = in.far;
    const long long step0 = in.step, since0 = in.since;
    if (threadIdx.x == 0) {
        int need = 0;
        int errn = err0;
        if (misplaced && err == 0) errn |= kErrInternal;
        if (close0) errn |= kErrClose;
        if (errn != err0) C->error = errn;
        if (close0) C->close_flag = 0;
        if (active && !init) {
            C->steps_left = left - 1;
            C->step = step0 + 1;
            C->since_reorder = since0 + 1;
            if (!last) {
                C->parity = par ^ 1;
                // the rebuild decision of decide_rebuild, on the values read above
                need = (far0 != 0u) || a.cell_list_only;
                C->rebuild_flag = need;
                C->reorder_now = need && a.reorder_interval > 0 && since0 + 1 >= a.reorder_interval;
            } else {
                C->rebuild_flag = 0;
            }
            C->far_flag = 0u;
        } else if (!init) {
            C->far_flag = 0u;
        }
        C->d2max = d2;
        C->reach = shell_reach(a, d2);
        // a step that waited for its rebuild leaves it due
        if (!active && !init && in.pend && errn == 0) need = 1;
        if (has_next) cudaGraphSetConditional(next, need ? 1u : 0u);
        C->ticket = 0;
    }
}

// The step's closing work as a node of its own (one warp), run after the
// step kernel: the step's blocks then end without a block barrier or a
// ticket, and the serial tail leaves the step kernel.  It sees the counters
// the step's blocks saw (only this kernel changes them during a step).
template <class P, bool kFinal>
__global__ void k_step_tail(Args<P> a, int mode, cudaGraphConditionalHandle next, int has_next) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    // every counter and displacement bucket is requested at once: the
    // kernel is one round trip to L2 and the writes
    const CloseIn in = read_close_in(a.ctr);
    const unsigned d2 = d2_gather_warp(a);
    const bool init = kFinal && (mode == kModeInit);
    const bool last = kFinal && !init && in.left == 1;
    const bool misplaced = !kFinal && in.left == 1;
    const bool active = init || (in.err == 0 && in.left > 0 && !misplaced && !in.pend);
    close_step<P>(a, in, d2, in.err, in.left, in.par, init, last, misplaced, active, next, has_next);
}

// Profiling aid, not part of a step: adds to ctr->list_reads the number of
// list entries the next step will read (list_count at the current shell
// reach, summed over the atoms).
template <class P>
__global__ void __launch_bounds__(kBlock) k_count_reads(Args<P> a) {
    __shared__ double shs[kBlock / 32];
    const int64_t i = gtid();
    int c = 0;
    if (i < a.n && !a.cell_list_only) c = list_count(a, i, a.ctr->reach);
    const double s = block_sum((double)c, shs);
    if (threadIdx.x == 0) atomicAdd((unsigned long long*)&a.ctr->list_reads, (unsigned long long)s);
}

// Step (f) of Sec. 3.1: v <- s v (the product in FP64, stored in the
// velocity precision), and this block's KE partial of the new velocities
// (PE and W partials are those of the last final step and stay).
template <class P>
__global__ void __launch_bounds__(kBlock) k_rescale(Args<P> a, double s) {
    __shared__ double shs[kBlock / 32];
    using vel = typename P::vel;
    const int64_t i = gtid();
    double ke = 0.0;
    if (i < a.n) {
        vel* v[3] = {a.vx, a.vy, a.vz};
        for (int d = 0; d < 3; d++) {
            double x;
            if constexpr (P::kFp64) x = v[d][i] * s;
            else x = cvt::f64(v[d][i]) * s;
            vel y;
            if constexpr (P::kFp64) y = x;
            else y = cvt::f32(x);
            v[d][i] = y;
            double dy;
            if constexpr (P::kFp64) dy = y;
            else dy = cvt::f64(y);
            ke += dy * dy;
        }
        ke *= 0.5;
    }
    const double bk = block_sum(ke, shs);
    if (threadIdx.x == 0) a.part[3 * blockIdx.x + 0] = bk;
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
    unpack_cell(a.cell[i], cc[0], cc[1], cc[2]);
    const typename P::real* pb[3] = {a.pbx, a.pby, a.pbz};
    const double* o[3] = {a.ox, a.oy, a.oz};
    const typename P::vel* v[3] = {a.vx, a.vy, a.vz};
    for (int d = 0; d < 3; d++) {
        a.io_pos[3 * (int64_t)u + d] = abs_coord(a, d, cc[d], full_offset(pb[d][i], o[d][i]));
        if constexpr (P::kFp64) a.io_vel[3 * (int64_t)u + d] = v[d][i];
        else a.io_vel[3 * (int64_t)u + d] = cvt::f64(v[d][i]);
    }
}

template <class P>
__global__ void __launch_bounds__(kBlock) k_get_forces(Args<P> a, double* out) {
    int64_t i = gtid();
    if (i >= a.n) return;
    int64_t u = a.perm[i];
    if constexpr (P::kFp64) {
        out[3 * u + 0] = a.fx[i];
        out[3 * u + 1] = a.fy[i];
        out[3 * u + 2] = a.fz[i];
    } else {
        out[3 * u + 0] = cvt::f64(a.fx[i]);
        out[3 * u + 1] = cvt::f64(a.fy[i]);
        out[3 * u + 2] = cvt::f64(a.fz[i]);
    }
}

template <class P>
__global__ void __launch_bounds__(kBlock) k_get_cells(Args<P> a, int* out) {
    int64_t i = gtid();
    if (i >= a.n) return;
    out[a.perm[i]] = linear_of_packed(a.cell[i], a.G);
}

// Compares the FP32/integer-pipe conversions with the hardware conversions
// on hashed bit patterns spanning the magnitudes the step uses.  fails[k]
// counts mismatches of f64, f32, the fixed-point accumulation and from_fix.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class P>
__global__ void __launch_bounds__(kBlock) k_selftest(long long n, unsigned long long* fails) {
    long long t = gtid();
    if (t >= n) return;
    unsigned long long r = mix64((unsigned long long)t);
    unsigned long long r2 = mix64(r);
    // binary32 with exponent in [2^-100, 2^60), random sign and mantissa
    unsigned e32 = 27u + (unsigned)(r % 160u);
    float x = __uint_as_float((unsigned)((r >> 8) & 0x807FFFFFu) | (e32 << 23));
    if (__double_as_longlong(cvt::f64(x)) != __double_as_longlong((double)x)) atomicAdd(&fails[0], 1ull);
    // binary64 inside the binary32 normal range
    unsigned long long e64 = 1023ull - 120ull + (r2 % 240ull);
    double d = __longlong_as_double((long long)((r2 & 0x800FFFFFFFFFFFFFull) | (e64 << 52)));
    if (__float_as_uint(cvt::f32(d)) != __float_as_uint(__double2float_rn(d))) atomicAdd(&fails[1], 1ull);
    // fixed point: g with |g| in [2^-40, 2^30); g and -g cancel exactly
    float g = __uint_as_float((unsigned)((r >> 16) & 0x807FFFFFu) | ((87u + (unsigned)(r2 % 70u)) << 23));
    Fix one, both;
    one.add(g);
    both.add(g);
    both.add(-g);
    long long ref = __float2ll_rn(g * 4294967296.0f);  // the product is exact
    if (one.value() != ref || both.value() != 0) atomicAdd(&fails[2], 1ull);
    long long qq = (long long)(r2 >> (r % 64u)) * ((r & 1u) ? -1 : 1);
    if (__float_as_uint(cvt::from_fix(qq)) != __float_as_uint(__ll2float_rn(qq))) atomicAdd(&fails[3], 1ull);
}

// ---------------------------------------------------------------------------
// ensembles: independent replicas, one thread block (or one cluster) each
// ---------------------------------------------------------------------------

// The blocks that work on one replica: one thread block, or every block of
// a thread-block cluster (rank 0 leads).  Barriers between phases are block
// barriers or cluster barriers (hardware barrier.cluster: no polling).
struct Team {
    int rank, size;
    __device__ __forceinline__ bool lead_block() const { return rank == 0; }
    __device__ __forceinline__ bool leader() const { return rank == 0 && threadIdx.x == 0; }
    __device__ __forceinline__ int64_t first(int64_t per_block = 0) const {
        return (int64_t)rank * blockDim.x + threadIdx.x;
    }
    __device__ __forceinline__ int64_t stride() const { return (int64_t)size * blockDim.x; }
    __device__ __forceinline__ void sync() const {
        if (size > 1) {
            asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        } else {
            __syncthreads();
        }
    }
};

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Reads an int from the shared memory of block `rank` of this cluster.
__device__ __forceinline__ int cluster_load_shared(const int* local, unsigned rank) {
    unsigned a = (unsigned)__cvta_generic_to_shared(local), ra, v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
    return (int)v;
}

// Per-block scratch of the per-replica engine.
struct EnsShared {
    int maxv, job;
    long long entries;
    int carry;
    int warp_tot[32];
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Profiling aid: keeps the GPU busy for about ns nanoseconds (at most 2^20
// clock reads), so that the events queued after it are not timestamped
// before the host has queued the kernels they bracket.
template <class P>
__global__ void k_spin(long long ns) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long t0 = globaltimer_ns();
    for (int k = 0; k < (1 << 20); k++)
        if (globaltimer_ns() - t0 >= (unsigned long long)ns) break;
}

// Exclusive scan of the replica's cell counts into cell_start, by one block,
// and the largest occupancy (the paper's N_l) into C->max_occ.
template <class P>
__device__ __noinline__ void ens_scan(const Args<P>& a, EnsShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        sh.carry = 0;
        sh.maxv = 0;
    }
    int mx = 0;
    __syncthreads();
    for (int base = 0; base < a.ncells; base += blockDim.x) {
        const int c = base + threadIdx.x;
        const int v = c < a.ncells ? a.count[c] : 0;
        mx = max(mx, v);
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sh.warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int t = lane < nw ? sh.warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            sh.warp_tot[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        const int excl = x - v + (warp > 0 ? sh.warp_tot[warp - 1] : 0) + sh.carry;
        if (c < a.ncells) a.cell_start[c] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) sh.carry = excl + v;
        __syncthreads();
    }
    atomicMax(&sh.maxv, mx);
    __syncthreads();
    if (threadIdx.x == 0) {
        a.cell_start[a.ncells] = (int)a.n;
        Counters* C = a.ctr;
        C->max_occ = sh.maxv;
        C->max_nn = 0;
        C->list_entries = 0;
    }
}

// The rebuild branch of one replica (the kernels k_bin .. k_rebuild_done,
// with team barriers between the phases).  stage: the block's dynamic
// shared memory, kEnsBuildStage 8-byte words per thread for the build.
template <class P>
__device__ __noinline__ void ens_rebuild(const Args<P>& a, EnsShared& sh, int* stage, Team tm) {
    Counters* C = a.ctr;
    const int64_t n = a.n, t0 = tm.first(), dt = tm.stride();
    for (int64_t i = t0; i < n; i += dt) bin_item<P>(a, i);
    tm.sync();
    if (tm.lead_block()) ens_scan<P>(a, sh);
    tm.sync();
    for (int64_t t = t0; t < n; t += dt) scatter_item<P>(a, t);
    for (int64_t c = t0; c < a.ncells; c += dt) a.count[c] = 0;
    tm.sync();
    for (int64_t c = t0; c < a.ncells; c += dt) cellsort_item<P>(a, c);
    tm.sync();
    for (int64_t s = t0; s < n; s += dt) gather_item<P>(a, s);
    tm.sync();
    if (C->reorder_now) {
        for (int64_t s = t0; s < n; s += dt) commit_item<P>(a, s);
        tm.sync();
    }
    int mx = 0;
    long long sum = 0;
    for (int64_t s = t0; s < n; s += dt) {
        const int m = build_item<P, false, kEnsBuildStage>(a, s, reinterpret_cast<int2*>(stage) + threadIdx.x,
                                                           (int)blockDim.x);
        mx = max(mx, m);
        sum += m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&C->max_nn, mx);
        atomicAdd((unsigned long long*)&C->list_entries, (unsigned long long)sum);
    }
    tm.sync();
    if (tm.leader()) {
        C->rebuilds += 1;
        if (C->reorder_now) {
            C->reorders += 1;
            C->since_reorder = 0;
            C->reorder_now = 0;
        }
        C->rebuild_flag = 0;
        C->d2max = 0u;
    }
    tm.sync();
}

// One step of one replica (k_step): warps take 32 atoms at a time, stage
// their list rows, compute forces and integrate; then the counters advance
// as in k_step's last block.  kFinal: the init or last step, whose KE, PE
// and W are summed over 32-atom chunks in a fixed order.
template <class P, bool kFinal>
__device__ __noinline__ void ens_step(const Args<P>& a, int* rows, bool init, Team tm) {
    Counters* C = a.ctr;
    const int err = C->error;
    const long long left = C->steps_left;
    const int par = C->parity;
    const bool last = kFinal && !init && left == 1;
    const bool active = init || (err == 0 && left > 0);
    const bool energy = init || last;
    const typename P::pos4* pc = par ? a.pB : a.pA;
    typename P::pos4* pn = par ? a.pA : a.pB;
    // read past L1: other blocks of the team raised it in the last step
    const int reach = shell_reach(a, __ldcg(&C->d2max));
    bool far = false, close = false;
    unsigned d2m = 0u;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t nchunks = (a.n + 31) / 32;
    for (int64_t ch = (int64_t)tm.rank * nw + (threadIdx.x >> 5); ch < nchunks; ch += (int64_t)tm.size * nw) {
        const int64_t i = ch * 32 + lane;
        int cnt, staged;
        const int* col;
        stage_rows<P, false>(a, i, reach, rows, cnt, staged, col);
        stage_wait<false>();
        bool f = false, cl = false;
        double k = 0.0, u = 0.0, w = 0.0;
        unsigned d2b = 0u;
        step_atom<P, false, kFinal>(a, i, i < a.n, active, init, energy, cnt, col, rows, staged, pc, pn, nullptr,
                                    nullptr, f, cl, k, u, w, d2b);
        far |= f;
        close |= cl;
        d2m = max(d2m, d2b);
        if (kFinal && energy) {  // fixed-shape sum over the chunk's 32 atoms
            for (int o = 16; o > 0; o >>= 1) {
                k += __shfl_xor_sync(0xffffffffu, k, o);
                u += __shfl_xor_sync(0xffffffffu, u, o);
                w += __shfl_xor_sync(0xffffffffu, w, o);
            }
            if (lane == 0) {
                a.part[3 * ch + 0] = k;
                a.part[3 * ch + 1] = u;
                a.part[3 * ch + 2] = w;
            }
        }
        __syncwarp();  // the next chunk's copies overwrite rows
    }
    if (__any_sync(0xffffffffu, far) && lane == 0) atomicOr(&C->far_flag, 1u);
    if (__any_sync(0xffffffffu, close) && lane == 0) atomicOr(&C->close_flag, 1);
    warp_max_into<true>(d2m, &C->d2max);
    tm.sync();
    if (kFinal && energy) {
        // chunk sums -> sums of 32 consecutive chunks (fixed shape, in any
        // warp) -> their sum in order: the same numbers whatever the launch
        const int64_t ngroups = (nchunks + 31) / 32;
        double* gsum = a.part + 3 * nchunks;
        for (int64_t g = (int64_t)tm.rank * nw + (threadIdx.x >> 5); g < ngroups; g += (int64_t)tm.size * nw) {
            const int64_t c = g * 32 + lane;
            double k = c < nchunks ? a.part[3 * c + 0] : 0.0;
            double u = c < nchunks ? a.part[3 * c + 1] : 0.0;
            double w = c < nchunks ? a.part[3 * c + 2] : 0.0;
            for (int o = 16; o > 0; o >>= 1) {
                k += __shfl_xor_sync(0xffffffffu, k, o);
                u += __shfl_xor_sync(0xffffffffu, u, o);
                w += __shfl_xor_sync(0xffffffffu, w, o);
            }
            if (lane == 0) {
                gsum[3 * g + 0] = k;
                gsum[3 * g + 1] = u;
                gsum[3 * g + 2] = w;
            }
        }
        tm.sync();
    }
    if (tm.leader()) {
        if (active && !init) {
            C->steps_left = left - 1;
            C->step += 1;
            C->since_reorder += 1;
            if (!last) {
                C->parity = par ^ 1;
                decide_rebuild(C, a.cell_list_only, a.reorder_interval);
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
        if (kFinal && energy && active) {
            const int64_t ngroups = (nchunks + 31) / 32;
            const double* gsum = a.part + 3 * nchunks;
            double k = 0.0, u = 0.0, w = 0.0;
            for (int64_t g = 0; g < ngroups; g++) {
                k += gsum[3 * g + 0];
                u += gsum[3 * g + 1];
                w += gsum[3 * g + 2];
            }
            C->ke = k;
            C->pe = u;
            C->virial = w;
        }
    }
    tm.sync();
}

// One job: load the replica's state when asked (md_set_state), then
// `nsteps` steps (md_step).  Every block of the team runs it.
template <class P>
__device__ __noinline__ void ens_job(const Args<P>& a, EnsShared& sh, int* smem, int init, long long nsteps,
                                     Team tm) {
    Counters* C = a.ctr;
    int* rows = smem + (threadIdx.x >> 5) * (kStageRows * 32);
    if (init) {
        if (tm.leader()) {
            Counters z = {};
            z.rebuild_flag = 1;
            z.reorder_now = 1;
            *C = z;
        }
        tm.sync();
        for (int64_t i = tm.first(); i < a.n; i += tm.stride()) set_state_item<P>(a, i);
        tm.sync();
        if (C->error == 0) ens_rebuild<P>(a, sh, smem, tm);
        if (C->error == 0) ens_step<P, true>(a, rows, true, tm);
    }
    if (nsteps > 0 && C->error == 0) {
        bool far = false;
        unsigned d2m = 0u;
        const int par = C->parity;
        for (int64_t i = tm.first(); i < a.n; i += tm.stride()) {
            unsigned d2b = 0u;
            far |= kickdrift_item<P>(a, i, par ? a.pB : a.pA, d2b);
            d2m = max(d2m, d2b);
        }
        if (__any_sync(0xffffffffu, far) && (threadIdx.x & 31) == 0) atomicOr(&C->far_flag, 1u);
        warp_max_into<true>(d2m, &C->d2max);
        tm.sync();
        if (tm.leader()) {
            C->steps_left = nsteps;
            decide_rebuild(C, a.cell_list_only, a.reorder_interval);
        }
        tm.sync();
        for (long long st = 0; st < nsteps; st++) {
            if (C->rebuild_flag) ens_rebuild<P>(a, sh, smem, tm);
            if (C->error) break;
            if (st + 1 < nsteps) ens_step<P, false>(a, rows, false, tm);
            else ens_step<P, true>(a, rows, false, tm);
            if (C->error) break;
        }
    }
    tm.sync();
}

template <class P>
__device__ __forceinline__ void ens_load_args(Args<P>& dst, const Args<P>* src) {
    static_assert(sizeof(Args<P>) % 16 == 0, "Args must be a whole number of 16-byte words");
    const int4* s4 = reinterpret_cast<const int4*>(src);
    int4* d4 = reinterpret_cast<int4*>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(Args<P>) / 16); k += blockDim.x) d4[k] = s4[k];
}

// The per-replica engine.  hdr = {queue[0], queue[1], njobs, nteam}, written
// by the host before each launch, so that one captured launch serves every
// run.  Jobs [0, nteam) -- the big replicas -- are run by whole clusters
// (when the launch has clusters of more than one block), taken from queue[0]
// by each cluster's first block; the remaining jobs are run by single blocks,
// taken from queue[1].  Both lists are in decreasing order of work.  Dynamic shared memory: kEnsSmemInts ints per thread (the
// step's staged rows, kStageRows x 32 per warp, or the build's staging).
template <class P>
__global__ void __launch_bounds__(1024, 1) k_ensemble(const Args<P>* __restrict__ reps, EnsJob* jobs, int* hdr) {
    int* queue = hdr;
    const int njobs = hdr[2], nteam = hdr[3];
    extern __shared__ __align__(16) int ens_smem[];
    __shared__ EnsShared sh;
    __shared__ __align__(16) Args<P> a;
    const unsigned cs = cluster_size();
    if (cs > 1) {
        const Team tm{(int)cluster_rank(), (int)cs};
        for (;;) {
            if (tm.leader()) sh.job = atomicAdd(&queue[0], 1);
            tm.sync();
            const int j = cluster_load_shared(&sh.job, 0);
            tm.sync();  // the first block keeps its slot until everyone has read it
            if (j >= nteam) break;
            ens_load_args<P>(a, reps + jobs[j].rep);
            if (tm.leader()) jobs[j].t_start = globaltimer_ns();
            tm.sync();
            ens_job<P>(a, sh, ens_smem, jobs[j].init, jobs[j].nsteps, tm);
            if (tm.leader()) jobs[j].t_end = globaltimer_ns();
        }
    }
    const Team solo{0, 1};
    for (;;) {
        if (threadIdx.x == 0) sh.job = nteam + atomicAdd(&queue[1], 1);
        __syncthreads();
        const int j = sh.job;
        if (j >= njobs) break;
        ens_load_args<P>(a, reps + jobs[j].rep);
        if (threadIdx.x == 0) jobs[j].t_start = globaltimer_ns();
        __syncthreads();
        ens_job<P>(a, sh, ens_smem, jobs[j].init, jobs[j].nsteps, solo);
        if (threadIdx.x == 0) jobs[j].t_end = globaltimer_ns();
        __syncthreads();
    }
    if (cs > 1) {  // no block leaves while another of its cluster may still address it
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
}

// ---------------------------------------------------------------------------
// kernel table used by the host runtime (graph nodes and eager launches)
// ---------------------------------------------------------------------------

template <class P>
KernelTable<P> make_kernel_table() {
    KernelTable<P> t;
    t.set_state = (void*)k_set_state<P>;
    t.bin = (void*)k_bin<P>;
    t.scan_apply = (void*)k_scan_apply<P>;
    t.scatter = (void*)k_scatter<P>;
    t.cellsort = (void*)k_cellsort<P>;
    t.gather = (void*)k_gather<P>;
    t.commit = (void*)k_commit<P>;
    t.build = (void*)k_build<P>;
    t.build_rows = (void*)k_build<P, true>;
    t.build_direct = (void*)k_build<P, false, true>;
    t.build_wc = (void*)k_build_wc<P>;
    t.rebuild_done = (void*)k_rebuild_done<P>;
    t.cond = (void*)k_cond<P>;
    t.kickdrift = (void*)k_kickdrift<P>;
    t.step_tail = (void*)k_step_tail<P, false>;
    t.step_tail_final = (void*)k_step_tail<P, true>;
    if constexpr (P::kFp64) t.step_list = (void*)k_step<P, false, false>;
    else t.step_list = (void*)k_step<P, false, false, kStepBlockMixed>;
    t.step_list_final = (void*)k_step<P, false, true>;
    t.step_cells = (void*)k_step<P, true, false>;
    t.step_cells_final = (void*)k_step<P, true, true>;
    t.finalize = (void*)k_finalize<P>;
    t.get_state = (void*)k_get_state<P>;
    t.get_forces = (void*)k_get_forces<P>;
    t.get_cells = (void*)k_get_cells<P>;
    t.reset_counters = (void*)k_reset_counters<P>;
    t.clear_overflow = (void*)k_clear_overflow<P>;
    t.selftest = (void*)k_selftest<P>;
    t.rescale = (void*)k_rescale<P>;
    t.count_reads = (void*)k_count_reads<P>;
    t.spin = (void*)k_spin<P>;
    if constexpr (!P::kFp64) {
        t.ensemble = (void*)k_ensemble<P>;
        // ablation variants of the mixed list form: {plain, final}
        t.step_var[0][0] = (void*)k_step<P, false, false, kStepBlockMixed, false, false>;  // plain loads
        t.step_var[0][1] = (void*)k_step<P, false, true, kBlock, false, false>;
        t.step_var[1][0] = (void*)k_step<P, false, false, kStepBlockMixed, true, true>;    // W transposed
        t.step_var[1][1] = (void*)k_step<P, false, true, kBlock, true, true>;
        t.step_var[2][0] = (void*)k_step<P, false, false, 64, true, false>;       // 64 threads per block
        t.step_var[2][1] = (void*)k_step<P, false, true, kBlock, true, false>;
        t.step_var[3][0] = (void*)k_step<P, false, false, 256, true, false>;      // 256 threads per block
        t.step_var[3][1] = (void*)k_step<P, false, true, kBlock, true, false>;
    } else {
        t.ensemble = nullptr;
        for (auto& v : t.step_var) v[0] = v[1] = nullptr;
    }
    return t;
}

}  // namespace md
