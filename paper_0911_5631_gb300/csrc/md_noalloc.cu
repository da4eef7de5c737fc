// md_noalloc.cu -- md_forces_noalloc: forces, potential energy and virial of
// one configuration with no device allocation at all.
//
// Who needs it: callers that may not allocate device memory themselves --
// code running inside a memory pool or budget it does not own, or on a
// path where cudaMalloc/cudaFree must not run because they synchronise the
// device and would stall other streams.  They pass input and output buffers;
// every working array lives in one fixed scratch area compiled into this
// library (a file-scope __device__ array), which each GPU that loads the
// library keeps until the process exits.
//
// The computation is the FP64 form of the pair-force step: wrap, bin into
// cells of width >= r_c (counting sort, deterministic order inside each
// cell), then forces from the 27 neighbouring cells with Eq. (1) plus the
// shift, and the sums U and W.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "../../include/md.h"

namespace md {
// Records the message md_last_error(NULL) returns (defined with the rest of
// the C ABI; not exported).
void set_call_error(const char* msg);
}  // namespace md

namespace {

constexpr int kThreads = 256;
constexpr int kMaxAtoms = MD_NOALLOC_MAX_ATOMS;
constexpr int kMaxCells = MD_NOALLOC_MAX_CELLS;
constexpr int kMaxBlocks = (kMaxAtoms + kThreads - 1) / kThreads;

// Byte layout of the scratch area.
constexpr size_t kOffCount = 0;                                            // int[kMaxCells]
constexpr size_t kOffStart = kOffCount + sizeof(int) * kMaxCells;          // int[kMaxCells + 1]
constexpr size_t kOffCell = kOffStart + sizeof(int) * (kMaxCells + 64);    // int[kMaxAtoms]
constexpr size_t kOffRank = kOffCell + sizeof(int) * kMaxAtoms;            // int[kMaxAtoms]
constexpr size_t kOffOrder = kOffRank + sizeof(int) * kMaxAtoms;           // int[kMaxAtoms]
constexpr size_t kOffPart = kOffOrder + sizeof(int) * kMaxAtoms;           // double[2 kMaxBlocks]
constexpr size_t kOffPos = (kOffPart + sizeof(double) * 2 * kMaxBlocks + 255) & ~size_t(255);  // double4[kMaxAtoms]
constexpr size_t kOffFlag = kOffPos + sizeof(double) * 4 * kMaxAtoms;     // int: a non-finite input was seen
constexpr size_t kScratchBytes = kOffFlag + 256;
static_assert(kScratchBytes <= MD_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the declared size");

__device__ __align__(256) unsigned char g_scratch[MD_NOALLOC_SCRATCH_BYTES];

struct Geo {
    int n, ncells;
    int G[3];
    double L[3], hL[3], invL[3], invW[3];
    double rc2, ushift;
};

struct Scratch {
    int* count;
    int* start;
    int* cell;
    int* rank;
    int* order;
    double* part;
    double* pos;  // x, y, z, index per atom in cell order
    int* bad;     // set when a position is not finite
};

__device__ __forceinline__ int gid() { return blockIdx.x * blockDim.x + threadIdx.x; }

// Wrap one component into [-L/2, L/2) and return its cell coordinate (same
// operation order as the handle-based path).
__device__ __forceinline__ int wrap_bin(double& x, const Geo& g, int d) {
    double s = floor(__dmul_rn(__dadd_rn(x, g.hL[d]), g.invL[d]));
    x = __dsub_rn(x, __dmul_rn(s, g.L[d]));
    int c = (int)floor(__dmul_rn(__dadd_rn(x, g.hL[d]), g.invW[d]));
    // a coordinate rounded onto a face belongs to the cell across it; move
    // it with its cell so the periodic shifts stay consistent
    if (c >= g.G[d]) { c -= g.G[d]; x = __dsub_rn(x, g.L[d]); }
    if (c < 0) { c += g.G[d]; x = __dadd_rn(x, g.L[d]); }
    if (c < 0 || c >= g.G[d]) c = 0;  // non-finite input; keeps indices in range
    return c;
}

__global__ void nz_zero(Geo g, Scratch s) {
    for (int c = gid(); c < g.ncells; c += gridDim.x * blockDim.x) s.count[c] = 0;
    if (gid() == 0) *s.bad = 0;
}

__global__ void nz_bin(Geo g, Scratch s, const double* __restrict__ pos) {
    int i = gid();
    if (i >= g.n) return;
    int c[3];
    bool finite = true;
    for (int d = 0; d < 3; d++) {
        double x = pos[3 * (size_t)i + d];
        finite = finite && isfinite(x);
        c[d] = wrap_bin(x, g, d);
    }
    if (!finite) atomicExch(s.bad, 1);
    int cl = (c[2] * g.G[1] + c[1]) * g.G[0] + c[0];
    s.cell[i] = cl;
    s.rank[i] = atomicAdd(&s.count[cl], 1);
}

// One block: exclusive scan of the counts (at most kMaxCells of them).
__global__ void nz_scan(Geo g, Scratch s) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < g.ncells; base += blockDim.x) {
        int idx = base + threadIdx.x;
        int v = idx < g.ncells ? s.count[idx] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        int excl = x - v + (warp > 0 ? warp_tot[warp - 1] : 0) + carry;
        if (idx < g.ncells) s.start[idx] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) s.start[g.ncells] = g.n;
}

__global__ void nz_scatter(Geo g, Scratch s) {
    int i = gid();
    if (i >= g.n) return;
    int slot = s.start[s.cell[i]] + s.rank[i];
    if (slot >= 0 && slot < g.n) s.order[slot] = i;
}

// Ascending atom index inside each cell (deterministic summation order).
__global__ void nz_sort(Geo g, Scratch s) {
    int c = gid();
    if (c >= g.ncells) return;
    int beg = s.start[c], end = s.start[c + 1];
    for (int k = beg + 1; k < end; k++) {
        int key = s.order[k];
        int t = k - 1;
        while (t >= beg && s.order[t] > key) {
            s.order[t + 1] = s.order[t];
            t--;
        }
        s.order[t + 1] = key;
    }
}

__global__ void nz_gather(Geo g, Scratch s, const double* __restrict__ pos) {
    int k = gid();
    if (k >= g.n) return;
    int i = s.order[k];
    double* q = s.pos + 4 * (size_t)k;
    for (int d = 0; d < 3; d++) {
        double x = pos[3 * (size_t)i + d];
        wrap_bin(x, g, d);
        q[d] = x;
    }
    q[3] = __longlong_as_double((long long)i);
}

// Forces on every atom from the 27 cells around its cell; per-block sums of
// 1/2 sum_j u and 1/2 sum_j r.f (each pair is seen from both atoms).
__global__ void nz_force(Geo g, Scratch s, double* __restrict__ f) {
    __shared__ double sh_u[kThreads / 32], sh_w[kThreads / 32];
    int k = gid();
    double uu = 0.0, ww = 0.0;
    if (k < g.n) {
        const double* qi = s.pos + 4 * (size_t)k;
        double xi = qi[0], yi = qi[1], zi = qi[2];
        int i = (int)__double_as_longlong(qi[3]);
        int cl = s.cell[i];
        int cx = cl % g.G[0], cy = (cl / g.G[0]) % g.G[1], cz = cl / (g.G[0] * g.G[1]);
        double fx = 0.0, fy = 0.0, fz = 0.0;
        for (int dz = -1; dz <= 1; dz++) {
            int z = cz + dz;
            double bz = 0.0;
            if (z >= g.G[2]) { z -= g.G[2]; bz = -g.L[2]; }
            if (z < 0) { z += g.G[2]; bz = g.L[2]; }
            for (int dy = -1; dy <= 1; dy++) {
                int y = cy + dy;
                double by = 0.0;
                if (y >= g.G[1]) { y -= g.G[1]; by = -g.L[1]; }
                if (y < 0) { y += g.G[1]; by = g.L[1]; }
                for (int dx = -1; dx <= 1; dx++) {
                    int x = cx + dx;
                    double bx = 0.0;
                    if (x >= g.G[0]) { x -= g.G[0]; bx = -g.L[0]; }
                    if (x < 0) { x += g.G[0]; bx = g.L[0]; }
                    int c2 = (z * g.G[1] + y) * g.G[0] + x;
                    int beg = s.start[c2], end = min(s.start[c2 + 1], g.n);
                    for (int t = beg; t < end; t++) {
                        if (t == k) continue;
                        const double* qj = s.pos + 4 * (size_t)t;
                        double ex = (xi - qj[0]) + bx;
                        double ey = (yi - qj[1]) + by;
                        double ez = (zi - qj[2]) + bz;
                        double r2 = ex * ex + ey * ey + ez * ez;
                        if (r2 < g.rc2) {
                            double ir2 = 1.0 / r2;
                            double ir6 = ir2 * ir2 * ir2;
                            double fr = 48.0 * ir6 * (ir6 - 0.5) * ir2;
                            fx += fr * ex;
                            fy += fr * ey;
                            fz += fr * ez;
                            uu += 4.0 * ir6 * (ir6 - 1.0) + g.ushift;
                            ww += fr * r2;
                        }
                    }
                }
            }
        }
        f[3 * (size_t)i + 0] = fx;
        f[3 * (size_t)i + 1] = fy;
        f[3 * (size_t)i + 2] = fz;
    }
    uu *= 0.5;
    ww *= 0.5;
    for (int o = 16; o > 0; o >>= 1) {
        uu += __shfl_xor_sync(0xffffffffu, uu, o);
        ww += __shfl_xor_sync(0xffffffffu, ww, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh_u[threadIdx.x >> 5] = uu;
        sh_w[threadIdx.x >> 5] = ww;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double su = 0.0, sw = 0.0;
        for (int w = 0; w < kThreads / 32; w++) {
            su += sh_u[w];
            sw += sh_w[w];
        }
        s.part[2 * blockIdx.x + 0] = su;
        s.part[2 * blockIdx.x + 1] = sw;
    }
}

__global__ void nz_reduce(int nblocks, Scratch s, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double su = 0.0, sw = 0.0;
        for (int b = 0; b < nblocks; b++) {
            su += s.part[2 * b + 0];
            sw += s.part[2 * b + 1];
        }
        out[0] = su;
        out[1] = sw;
    }
}

// Address of g_scratch on the current device.  Looked up on every call (a
// cheap query): a cached address would go stale if the caller reset the
// device and the module were loaded again.
int scratch_for_current_device(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        md::set_call_error("no current CUDA device");
        return MD_ENODEV;
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        md::set_call_error((std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
        return MD_ECUDA;
    }
    *out = p;
    return MD_OK;
}

}  // namespace

extern "C" int md_forces_noalloc(const double box[3], int64_t n, double rc, double ushift, const double* pos,
                                 double* f, double* pe_vir, void* stream) {
    if (!box || !pos || !f || !pe_vir) {
        md::set_call_error("NULL argument");
        return MD_EINVAL;
    }
    if (n <= 0 || n > kMaxAtoms) {
        md::set_call_error("n must be in [1, MD_NOALLOC_MAX_ATOMS]");
        return MD_EINVAL;
    }
    if (!(rc > 0.0) || !std::isfinite(rc)) {
        md::set_call_error("rc must be positive and finite");
        return MD_EINVAL;
    }
    Geo g;
    std::memset(&g, 0, sizeof(g));
    g.n = (int)n;
    int64_t nc = 1;
    for (int d = 0; d < 3; d++) {
        if (!(box[d] > 0.0) || !std::isfinite(box[d])) {
            md::set_call_error("box edges must be positive and finite");
            return MD_EINVAL;
        }
        double gd = std::floor(box[d] / rc);
        if (gd < 3.0) {
            md::set_call_error("box edge below 3 r_c: the 27-cell neighbourhood would alias");
            return MD_EINVAL;
        }
        if (gd > (double)kMaxCells) gd = (double)kMaxCells;
        g.G[d] = (int)gd;
        nc *= g.G[d];
        g.L[d] = box[d];
        g.hL[d] = 0.5 * box[d];
        g.invL[d] = 1.0 / box[d];
        g.invW[d] = (double)g.G[d] / box[d];
    }
    if (nc > kMaxCells) {
        md::set_call_error("more cells than MD_NOALLOC_MAX_CELLS (box too large for r_c)");
        return MD_EINVAL;
    }
    g.ncells = (int)nc;
    g.rc2 = rc * rc;
    if (std::isnan(ushift)) ushift = std::fabs(rc - std::pow(2.0, 1.0 / 6.0)) <= 1e-12 * rc ? 1.0 : 0.0;
    g.ushift = ushift;

    void* base = nullptr;
    int r = scratch_for_current_device(&base);
    if (r) return r;
    unsigned char* b = (unsigned char*)base;
    Scratch s;
    s.count = (int*)(b + kOffCount);
    s.start = (int*)(b + kOffStart);
    s.cell = (int*)(b + kOffCell);
    s.rank = (int*)(b + kOffRank);
    s.order = (int*)(b + kOffOrder);
    s.part = (double*)(b + kOffPart);
    s.pos = (double*)(b + kOffPos);
    s.bad = (int*)(b + kOffFlag);

    cudaStream_t st = (cudaStream_t)stream;
    int ga = (g.n + kThreads - 1) / kThreads;
    int gc = (g.ncells + kThreads - 1) / kThreads;
    nz_zero<<<gc, kThreads, 0, st>>>(g, s);
    nz_bin<<<ga, kThreads, 0, st>>>(g, s, pos);
    nz_scan<<<1, 1024, 0, st>>>(g, s);
    nz_scatter<<<ga, kThreads, 0, st>>>(g, s);
    nz_sort<<<gc, kThreads, 0, st>>>(g, s);
    nz_gather<<<ga, kThreads, 0, st>>>(g, s, pos);
    nz_force<<<ga, kThreads, 0, st>>>(g, s, f);
    nz_reduce<<<1, 32, 0, st>>>(ga, s, pe_vir);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        md::set_call_error((std::string("launch: ") + cudaGetErrorString(e)).c_str());
        return MD_ECUDA;
    }
    // the non-finite check: a 4-byte read of the flag into this stack
    // variable, after the call's own work on the stream
    int bad = 0;
    e = cudaMemcpyAsync(&bad, s.bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        md::set_call_error((std::string("flag read: ") + cudaGetErrorString(e)).c_str());
        return MD_ECUDA;
    }
    if (bad) {
        md::set_call_error("non-finite position");
        return MD_EUNSTABLE;
    }
    return MD_OK;
}
