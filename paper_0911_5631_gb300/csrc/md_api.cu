// md_api.cu -- host runtime and C ABI of libmd (declared in include/md.h).
//
// A handle owns the device state of one simulation and a CUDA stream.  One
// md_step call enqueues: the half kick + drift of the first step, then the
// steps themselves.  With graphs enabled the steps run as replays of a
// CUDA graph holding K (force + integrate, closing) pairs with a conditional
// rebuild node before every third step; the closing kernel decides on the
// device whether the next rebuild branch runs (cudaGraphSetConditional), so
// no host round trip sits inside the loop, and a step whose rebuild is due
// before the next conditional node waits (the call runs it at its end).
// Without graphs the same kernels are launched one by one and the host
// reads the rebuild flag before each step.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/md.h"
#include "md_common.cuh"

#include "md_table.h"
#include "md_host.h"

namespace {

using namespace md;

thread_local std::string g_create_error;

constexpr int kChunk = 32;  // steps per graph replay

// Zeroed storage for cudaGraphNodeParams (its union has no default
// constructor).
struct NodeParams {
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    NodeParams() { std::memset(raw, 0, sizeof(raw)); }
    cudaGraphNodeParams& get() { return *reinterpret_cast<cudaGraphNodeParams*>(raw); }
};

struct DevGuard {
    int prev = -1;
    bool changed = false;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) changed = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DevGuard() {
        if (changed && prev >= 0) cudaSetDevice(prev);
    }
};

struct SimBase {
    virtual ~SimBase() {}
    virtual int set_state(const double* pos, const double* vel, bool device) = 0;
    virtual int step(int64_t n) = 0;
    virtual int rescale(double T) = 0;
    virtual int measure(md_measure_t* out) = 0;
    virtual int get_state(double* pos, double* vel, bool device) = 0;
    virtual int get_forces(double* f) = 0;
    virtual int debug_cells(int32_t* cell) = 0;
    virtual int debug_neighbors(int64_t* count, int64_t* entries, int32_t* pairs, int64_t cap) = 0;
    virtual int get_plan(md_plan_t* out) = 0;
    virtual int set_profiling(int on) = 0;
    virtual int kernel_stats(md_kernel_stats_t* out) = 0;
    virtual int sync() = 0;
    std::string err;
    int device = 0;
};

#define MD_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                    \
            return e_ == cudaErrorMemoryAllocation ? MD_ENOMEM : MD_ECUDA;               \
        }                                                                                \
    } while (0)

template <class P>
struct Sim : SimBase {
    using real = typename P::real;
    using vel = typename P::vel;
    using pos4 = typename P::pos4;

    Args<P> a{};
    KernelTable<P> kt{};
    md_params prm{};
    md_plan_t plan{};
    double box[3] = {0, 0, 0};
    double rc = 0, skin = 0, dt = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool have_state = false;
    std::vector<void*> allocs;
    int* nbr_alloc = nullptr;

    struct Chunk {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t e = nullptr;
        int K = 0;
    };
    Chunk big, one;
    bool graphs_ok = false;

    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    int64_t launches = 0;
    int64_t graph_launches = 0;
    int64_t steps_run = 0;
    int64_t rebuilds_at_mark = 0;
    double step_ms = 0.0;
    int64_t step_launches = 0;
    double rebuild_ms = 0.0;
    int64_t rebuilds_timed = 0;
    int64_t step_atoms = 0;
    int64_t step_bytes = 0;

    ~Sim() override {
        DevGuard dg(device);
        destroy_graphs();
        for (auto e : ev) cudaEventDestroy(e);
        for (void* p : allocs) cudaFree(p);
        if (nbr_alloc) cudaFree(nbr_alloc);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }

    template <class T>
    int alloc(T** p, size_t count) {
        void* q = nullptr;
        MD_CUDA(cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16));
        allocs.push_back(q);
        *p = (T*)q;
        return MD_OK;
    }

    int create(const double bx[3], int64_t n, double rc_, double skin_, double dt_, const md_params* p) {
        md_default_params(&prm);
        if (p) prm = *p;
        for (int k = 0; k < 3; k++) box[k] = bx[k];
        rc = rc_;
        skin = skin_;
        dt = dt_;
        int rcode = resolve_plan(bx, n, rc, skin, dt, &prm, &plan, &err);
        if (rcode) return rcode;
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            cudaGetLastError();
            err = "no CUDA device";
            return MD_ENODEV;
        }
        if (prm.device >= ndev) {
            err = "device ordinal out of range";
            return MD_EINVAL;
        }
        if (prm.device >= 0) device = prm.device;
        else MD_CUDA(cudaGetDevice(&device));
        DevGuard dg(device);
        if (prm.stream) {
            stream = (cudaStream_t)prm.stream;
        } else {
            MD_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
            own_stream = true;
        }
        kt = make_kernel_table<P>();
        fill_scalars(n);
        int r = allocate();
        if (r) return r;
        return MD_OK;
    }

    void fill_scalars(int64_t n) {
        fill_args_scalars(a, plan, box, n, rc, skin, dt, prm.cell_list_only, prm.reorder_interval, prm.shell_bins);
        a.list_rows = prm.variant == MD_VARIANT_LIST_ROWS;
    }

    int allocate() {
        int64_t n = a.n;
        int r = 0;
        auto chk = [&](int rr) { if (rr && !r) r = rr; };
        chk(alloc(&a.cell, n)); chk(alloc(&a.perm, n)); chk(alloc(&a.rank, n));
        chk(alloc(&a.pbx, n)); chk(alloc(&a.pby, n)); chk(alloc(&a.pbz, n));
        chk(alloc(&a.ox, n)); chk(alloc(&a.oy, n)); chk(alloc(&a.oz, n));
        chk(alloc(&a.vx, n)); chk(alloc(&a.vy, n)); chk(alloc(&a.vz, n));
        chk(alloc(&a.fx, n)); chk(alloc(&a.fy, n)); chk(alloc(&a.fz, n));
        chk(alloc(&a.pA, pair_slots(n))); chk(alloc(&a.pB, pair_slots(n))); chk(alloc(&a.cand, n));
        chk(alloc(&a.s_cell, n)); chk(alloc(&a.s_perm, n));
        chk(alloc(&a.s_pbx, n)); chk(alloc(&a.s_pby, n)); chk(alloc(&a.s_pbz, n));
        chk(alloc(&a.s_ox, n)); chk(alloc(&a.s_oy, n)); chk(alloc(&a.s_oz, n));
        chk(alloc(&a.s_vx, n)); chk(alloc(&a.s_vy, n)); chk(alloc(&a.s_vz, n));
        chk(alloc(&a.count, a.ncells)); chk(alloc(&a.cell_start, (size_t)a.ncells + 1));
        chk(alloc(&a.order, n)); chk(alloc(&a.tile_sum, a.ntiles));
        chk(alloc(&a.nn, n)); chk(alloc(&a.lim, (size_t)(kShellBins - 1) * n));
        chk(alloc(&a.part, (size_t)3 * a.nblocks));
        chk(alloc(&a.ctr, 1));
        chk(alloc(&a.d2b, (size_t)kD2Buckets * 32));
        chk(alloc(&a.io_pos, (size_t)3 * n)); chk(alloc(&a.io_vel, (size_t)3 * n));
        if (r) return r;
        r = alloc_nbr(a.cap);
        if (r) return r;
        MD_CUDA(cudaMemsetAsync(a.count, 0, sizeof(int) * a.ncells, stream));
        MD_CUDA(cudaMemsetAsync(a.tile_sum, 0, sizeof(int) * a.ntiles, stream));
        MD_CUDA(cudaMemsetAsync(a.ctr, 0, sizeof(Counters), stream));
        MD_CUDA(cudaMemsetAsync(a.d2b, 0, sizeof(unsigned) * kD2Buckets * 32, stream));
        MD_CUDA(cudaMemsetAsync(a.nn, 0, sizeof(int) * n, stream));
        MD_CUDA(cudaStreamSynchronize(stream));
        return MD_OK;
    }

    int alloc_nbr(int cap) {
        if (nbr_alloc) {
            cudaFree(nbr_alloc);
            nbr_alloc = nullptr;
        }
        size_t cols = (size_t)((a.n + 31) / 32) * 32;
        size_t cnt = cols * (size_t)(cap > 0 ? cap : 1);
        void* q = nullptr;
        MD_CUDA(cudaMalloc(&q, cnt * sizeof(int)));
        nbr_alloc = (int*)q;
        a.nbr = nbr_alloc;
        a.cap = cap;
        plan.nbr_capacity = cap;
        return MD_OK;
    }

    // ---- launches ------------------------------------------------------

    template <class... T>
    cudaError_t launch(void* f, unsigned grid, unsigned block, T&... args) {
        void* p[] = {(void*)&args...};
        launches++;
        return cudaLaunchKernel(f, dim3(grid), dim3(block), p, 0, stream);
    }

    unsigned grid_atoms() const { return (unsigned)a.nblocks; }
    unsigned grid_cells() const { return (unsigned)((a.ncells + kBlock - 1) / kBlock); }
    unsigned grid_scatter() const {
        int64_t m = a.n > a.ncells ? a.n : a.ncells;
        return (unsigned)((m + kBlock - 1) / kBlock);
    }

    // the neighbour-list build: a block of kWcThreads per x slice of a
    // pencil (a warp per cell), or a thread per cell-ordered atom
    bool warp_build() const { return use_warp_build(prm); }
    void* build_fn() const {
        if (warp_build()) return kt.build_wc;
        if (a.list_rows) return kt.build_rows;
        return use_direct_build(box, a.n, plan.rn) ? kt.build_direct : kt.build;
    }
    unsigned grid_build() const {
        return warp_build() ? (unsigned)wc_slices(a) : (unsigned)((a.n + kBuildBlock - 1) / kBuildBlock);
    }
    unsigned block_build() const { return warp_build() ? (unsigned)kWcThreads : (unsigned)kBuildBlock; }

    // index into kt.step_var of the requested ablation variant, or -1
    int variant_index() const {
        switch (prm.variant) {
            case MD_VARIANT_PLAIN_LOADS: return 0;
            case MD_VARIANT_LIST_ROWS: return 1;
            case MD_VARIANT_BLOCK64: return 2;
            case MD_VARIANT_BLOCK256: return 3;
            default: return -1;
        }
    }
    void* step_fn(bool final_node) const {
        if (prm.cell_list_only) return final_node ? kt.step_cells_final : kt.step_cells;
        const int v = variant_index();
        if (v >= 0) return kt.step_var[v][final_node ? 1 : 0];
        return final_node ? kt.step_list_final : kt.step_list;
    }
    // threads per block of the step kernel (the final step always kBlock)
    unsigned step_block(bool final_node) const {
        if (final_node || P::kFp64 || prm.cell_list_only) return kBlock;
        if (prm.variant == MD_VARIANT_BLOCK64) return 64;
        if (prm.variant == MD_VARIANT_BLOCK256) return 256;
        return kStepBlockMixed;
    }
    unsigned step_grid(bool final_node) const {
        const unsigned b = step_block(final_node);
        return (unsigned)((a.n + b - 1) / b);
    }

    // The rebuild branch as stream launches.  guard = 1: every kernel returns
    // at once unless the device rebuild flag is set.
    int rebuild_eager(int g = 1) {
        MD_CUDA(launch(kt.bin, grid_atoms(), kBlock, a, g));
        MD_CUDA(launch(kt.scan_apply, (unsigned)a.ntiles, kBlock, a, g));
        MD_CUDA(launch(kt.scatter, grid_scatter(), kBlock, a, g));
        MD_CUDA(launch(kt.cellsort, grid_cells(), kBlock, a, g));
        MD_CUDA(launch(kt.gather, grid_atoms(), kBlock, a, g));
        MD_CUDA(launch(kt.commit, grid_atoms(), kBlock, a, g));
        if (!prm.cell_list_only) MD_CUDA(launch(build_fn(), grid_build(), block_build(), a, g));
        MD_CUDA(launch(kt.rebuild_done, 1, 32, a, g));
        return MD_OK;
    }

    // The step kernel, then (kStepTailNode) its one-warp closing kernel.
    // Profiling: the event `after_step` is recorded right after the step
    // kernel, and then the count of the entries that step read (before the
    // closing kernel changes the reach), so that the count kernel neither
    // falls inside the events nor warms the caches for the step.  A step
    // kernel that closes itself has its entries counted before it.
    int step_kernel_eager(int mode, bool final_node, cudaEvent_t after_step = nullptr) {
        cudaGraphConditionalHandle none = 0;
        int has = 0;
        MD_CUDA(launch(step_fn(final_node), step_grid(final_node), step_block(final_node), a, mode, none, has));
        if (after_step) {
            MD_CUDA(cudaEventRecord(after_step, stream));
            if (kStepTailNode) MD_CUDA(launch(kt.count_reads, grid_atoms(), kBlock, a));
        }
        if (kStepTailNode) MD_CUDA(launch(tail_fn(final_node), 1, 32, a, mode, none, has));
        return MD_OK;
    }
    void* tail_fn(bool final_node) const { return final_node ? kt.step_tail_final : kt.step_tail; }

    // ---- graphs ----------------------------------------------------------

    void destroy_graphs() {
        for (Chunk* c : {&big, &one}) {
            if (c->e) cudaGraphExecDestroy(c->e);
            if (c->g) cudaGraphDestroy(c->g);
            c->e = nullptr;
            c->g = nullptr;
            c->K = 0;
        }
        graphs_ok = false;
    }

    template <class... T>
    cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* dep, cudaGraphNode_t* out, void* f, unsigned grid,
                           unsigned block, T&... args) {
        void* p[] = {(void*)&args...};
        NodeParams buf;
        cudaGraphNodeParams& np = buf.get();
        np.type = cudaGraphNodeTypeKernel;
        np.kernel.func = f;
        np.kernel.gridDim = dim3(grid);
        np.kernel.blockDim = dim3(block);
        np.kernel.sharedMemBytes = 0;
        np.kernel.kernelParams = p;
        return cudaGraphAddNode(out, g, dep, nullptr, dep ? 1 : 0, &np);
    }

    int build_body(cudaGraph_t body) {
        int g = 0;
        cudaGraphNode_t prev = nullptr, cur = nullptr;
        auto chain = [&](cudaError_t e) -> cudaError_t {
            prev = cur;
            return e;
        };
        MD_CUDA(chain(add_kernel(body, nullptr, &cur, kt.bin, grid_atoms(), kBlock, a, g)));
        MD_CUDA(chain(add_kernel(body, &prev, &cur, kt.scan_apply, (unsigned)a.ntiles, kBlock, a, g)));
        MD_CUDA(chain(add_kernel(body, &prev, &cur, kt.scatter, grid_scatter(), kBlock, a, g)));
        MD_CUDA(chain(add_kernel(body, &prev, &cur, kt.cellsort, grid_cells(), kBlock, a, g)));
        MD_CUDA(chain(add_kernel(body, &prev, &cur, kt.gather, grid_atoms(), kBlock, a, g)));
        MD_CUDA(chain(add_kernel(body, &prev, &cur, kt.commit, grid_atoms(), kBlock, a, g)));
        if (!prm.cell_list_only)
            MD_CUDA(chain(add_kernel(body, &prev, &cur, build_fn(), grid_build(), block_build(), a, g)));
        MD_CUDA(chain(add_kernel(body, &prev, &cur, kt.rebuild_done, 1, 32, a, g)));
        return MD_OK;
    }

    // K steps: k_cond, then per step the step kernel and its closing kernel,
    // with a conditional rebuild node before every m-th step (every step in
    // the cell-list-only form, which rebuilds at each).  The closing kernel
    // before a conditional node sets its handle; a step after another whose
    // rebuild is due waits for the next conditional node.
    int build_chunk(Chunk& c, int K) {
        MD_CUDA(cudaGraphCreate(&c.g, 0));
        const int m = (prm.cell_list_only || a.n > kRebuildEveryMaxAtoms) ? 1 : kRebuildEvery;
        std::vector<cudaGraphConditionalHandle> h((K + m - 1) / m);
        for (auto& hh : h) MD_CUDA(cudaGraphConditionalHandleCreate(&hh, c.g, 0, 0));
        cudaGraphNode_t prev = nullptr, node = nullptr;
        MD_CUDA(add_kernel(c.g, nullptr, &node, kt.cond, 1, 32, a, h[0]));
        prev = node;
        int mode = kModeAuto;
        for (int s = 0; s < K; s++) {
            if (s % m == 0) {
                NodeParams buf;
                cudaGraphNodeParams& cp = buf.get();
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = h[s / m];
                cp.conditional.type = cudaGraphCondTypeIf;
                cp.conditional.size = 1;
                cudaGraphNode_t ifn = nullptr;
                MD_CUDA(cudaGraphAddNode(&ifn, c.g, &prev, nullptr, 1, &cp));
                int r = build_body(cp.conditional.phGraph_out[0]);
                if (r) return r;
                prev = ifn;
            }
            const int has = (s + 1 < K && (s + 1) % m == 0) ? 1 : 0;
            cudaGraphConditionalHandle nxt = has ? h[(s + 1) / m] : 0;
            // only a graph's last node can meet the last step of a call
            MD_CUDA(add_kernel(c.g, &prev, &node, step_fn(s + 1 == K), step_grid(s + 1 == K), step_block(s + 1 == K),
                               a, mode, nxt, has));
            if (kStepTailNode) {
                cudaGraphNode_t stepn = node;
                MD_CUDA(add_kernel(c.g, &stepn, &node, tail_fn(s + 1 == K), 1, 32, a, mode, nxt, has));
            }
            prev = node;
        }
        MD_CUDA(cudaGraphInstantiate(&c.e, c.g, 0));
        c.K = K;
        return MD_OK;
    }

    int ensure_graphs() {
        if (graphs_ok) return MD_OK;
        destroy_graphs();
        int r = build_chunk(big, kChunk);
        if (!r) r = build_chunk(one, 1);
        if (r) {
            destroy_graphs();
            return r;
        }
        graphs_ok = true;
        return MD_OK;
    }

    int graph_kernels_per_step() const { return 1; }

    // Enqueues nsteps (rebuild?, force + integrate) pairs.
    int run_steps(int64_t nsteps) {
        if (nsteps <= 0) return MD_OK;
        if (prm.use_graphs && !profiling) {
            int r = ensure_graphs();
            if (r) return r;
            int64_t nb = nsteps / kChunk, rem = nsteps % kChunk;
            for (int64_t b = 0; b < nb; b++) {
                MD_CUDA(cudaGraphLaunch(big.e, stream));
                graph_launches++;
                launches += 1 + kChunk * (kStepTailNode ? 2 : 1);
            }
            for (int64_t b = 0; b < rem; b++) {
                MD_CUDA(cudaGraphLaunch(one.e, stream));
                graph_launches++;
                launches += kStepTailNode ? 3 : 2;
            }
        } else {
            if (profiling && (int64_t)ev.size() < 4 * nsteps) {
                while ((int64_t)ev.size() < 4 * nsteps) {
                    cudaEvent_t e;
                    MD_CUDA(cudaEventCreate(&e));
                    ev.push_back(e);
                }
            }
            // Stream launches: the host reads the device rebuild flag before
            // each step, so only rebuilds that are due are launched (one
            // round trip per step; this path serves profiling and checks).
            std::vector<char> rebuilt(profiling ? nsteps : 0, 0);
            for (int64_t s = 0; s < nsteps; s++) {
                int flag = 0;
                MD_CUDA(cudaMemcpyAsync(&flag, &a.ctr->rebuild_flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
                MD_CUDA(cudaStreamSynchronize(stream));
                // the GPU waits on a short spin while the host queues the
                // bracketed kernels, so that no launch gap is timed
                long long spin_ns = 30000;
                if (profiling) MD_CUDA(launch(kt.spin, 1, 32, spin_ns));
                if (profiling && flag) {
                    rebuilt[s] = 1;
                    MD_CUDA(cudaEventRecord(ev[4 * s + 2], stream));
                }
                int r = flag ? rebuild_eager(0) : MD_OK;
                if (r) return r;
                if (profiling && flag) MD_CUDA(cudaEventRecord(ev[4 * s + 3], stream));
                if (profiling) {  // (the step closes itself: count before it)
                    if (!kStepTailNode) MD_CUDA(launch(kt.count_reads, grid_atoms(), kBlock, a));
                    MD_CUDA(cudaEventRecord(ev[4 * s], stream));
                }
                r = step_kernel_eager(kModeAuto, s + 1 == nsteps, profiling ? ev[4 * s + 1] : nullptr);
                if (r) return r;
            }
            if (profiling) {
                MD_CUDA(cudaStreamSynchronize(stream));
                for (int64_t s = 0; s < nsteps; s++) {
                    float ms = 0.f;
                    MD_CUDA(cudaEventElapsedTime(&ms, ev[4 * s], ev[4 * s + 1]));
                    step_ms += ms;
                    if (rebuilt[s]) {
                        MD_CUDA(cudaEventElapsedTime(&ms, ev[4 * s + 2], ev[4 * s + 3]));
                        rebuild_ms += ms;
                        rebuilds_timed++;
                    }
                }
                step_launches += nsteps;
                // algorithmic bytes: the per-atom state and the entries read
                Counters c;
                int rr = read_counters(&c);
                if (rr) return rr;
                MD_CUDA(cudaMemsetAsync(&a.ctr->list_reads, 0, sizeof(long long), stream));
                // per atom: pb, o, v, the new pair coordinate and the gathered
                // coordinates (116 B; 184 B in FP64), the list count (a byte
                // of lim with shell bins, else nn); the cells-only variant
                // keeps the 120 / 188 B of state and count of the list form
                const int64_t base = prm.cell_list_only ? (P::kFp64 ? 188 : 120)
                                                        : (P::kFp64 ? 184 : 116) + (prm.shell_bins ? 1 : 4);
                step_bytes += nsteps * base * a.n + 4 * c.list_reads;
            }
        }
        steps_run += nsteps;
        return MD_OK;
    }

    int read_counters(Counters* c) {
        MD_CUDA(cudaMemcpyAsync(c, a.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, stream));
        MD_CUDA(cudaStreamSynchronize(stream));
        return MD_OK;
    }

    int check_fatal(const Counters& c) {
        if (c.error & kErrInternal) {
            err = "internal: a step kernel without the final-step path met the last step of a call";
            return MD_ECUDA;
        }
        if (c.error & (kErrUnstable | kErrClose)) {
            err = (c.error & kErrClose) ? "two atoms came closer than the fixed-point force range allows"
                                        : "non-finite coordinate or velocity";
            return MD_EUNSTABLE;
        }
        return MD_OK;
    }

    // Enlarges the neighbour capacity after an overflow and rebuilds.
    int regrow(const Counters& c) {
        int need = c.need_cap > a.cap ? c.need_cap : a.cap + 4;
        int cap = (int)std::ceil(need * 1.25) + 4;
        cap = (cap + 3) & ~3;
        int cap_max = P::kFp64 ? 8192 : kMaxCapMixed;
        if (need > cap_max) {
            err = "an atom has more neighbours than the largest list capacity";
            return MD_EOVERFLOW;
        }
        if (cap > cap_max) cap = cap_max;
        MD_CUDA(cudaStreamSynchronize(stream));
        destroy_graphs();
        int r = alloc_nbr(cap);
        if (r) return r;
        MD_CUDA(launch(kt.clear_overflow, 1, 32, a.ctr));
        return rebuild_eager();
    }

    int finish_pending(int64_t* steps_left_out) {
        bool overflowed = false;
        for (int attempt = 0; attempt < 16; attempt++) {
            Counters c;
            int r = read_counters(&c);
            if (r) return r;
            r = check_fatal(c);
            if (r) return r;
            if (c.error & kErrOverflow) {
                overflowed = true;
                r = regrow(c);
                if (r) return r;
                // the step that met the overflow has not run yet
                Counters c2;
                r = read_counters(&c2);
                if (r) return r;
                if (c2.error & kErrOverflow) continue;
                r = run_steps(c2.steps_left);
                if (r) return r;
                continue;
            }
            if (c.steps_left > 0 && c.error == 0) {
                // steps that waited for a rebuild inside a graph: run them
                // now (each round leaves fewer to wait)
                r = run_steps(c.steps_left);
                if (r) return r;
                continue;
            }
            if (steps_left_out) *steps_left_out = c.steps_left;
            return MD_OK;
        }
        if (overflowed) {
            err = "neighbour list kept overflowing";
            return MD_EOVERFLOW;
        }
        err = "steps that waited for a rebuild did not complete";
        return MD_ECUDA;
    }

    // ---- API -------------------------------------------------------------

    int set_state(const double* pos, const double* vel, bool device) override {
        DevGuard dg(this->device);
        if (!pos || !vel) {
            err = "NULL state array";
            return MD_EINVAL;
        }
        size_t bytes = sizeof(double) * 3 * (size_t)a.n;
        cudaMemcpyKind k = device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        MD_CUDA(cudaMemcpyAsync(a.io_pos, pos, bytes, k, stream));
        MD_CUDA(cudaMemcpyAsync(a.io_vel, vel, bytes, k, stream));
        MD_CUDA(launch(kt.reset_counters, 1, 32, a.ctr));
        MD_CUDA(launch(kt.set_state, grid_atoms(), kBlock, a));
        int r = rebuild_eager();
        if (r) return r;
        for (int attempt = 0; attempt < 8; attempt++) {
            Counters c;
            r = read_counters(&c);
            if (r) return r;
            r = check_fatal(c);
            if (r) return r;
            if (!(c.error & kErrOverflow)) break;
            r = regrow(c);
            if (r) return r;
        }
        r = step_kernel_eager(kModeInit, true);
        if (r) return r;
        Counters c;
        r = read_counters(&c);
        if (r) return r;
        r = check_fatal(c);
        if (r) return r;
        have_state = true;
        return MD_OK;
    }

    int step(int64_t n) override {
        DevGuard dg(device);
        if (n <= 0) return MD_OK;
        if (!have_state) {
            err = "md_step before md_set_state";
            return MD_ESTATE;
        }
        long long nn = (long long)n;
        MD_CUDA(launch(kt.kickdrift, grid_atoms(), kBlock, a, nn));
        int r = run_steps(n);
        if (r) return r;
        int64_t left = 0;
        r = finish_pending(&left);
        if (r) return r;
        if (left != 0) {
            err = "step counter did not reach zero";
            return MD_ECUDA;
        }
        return MD_OK;
    }

    int rescale(double T) override {
        DevGuard dg(device);
        if (!have_state) {
            err = "md_rescale before md_set_state";
            return MD_ESTATE;
        }
        if (!(T > 0.0) || !std::isfinite(T)) {
            err = "T must be positive and finite";
            return MD_EINVAL;
        }
        MD_CUDA(launch(kt.finalize, 1, kBlock, a));
        Counters c;
        int r = read_counters(&c);
        if (r) return r;
        if (!(c.ke > 0.0)) {
            err = "kinetic energy is zero";
            return MD_EINVAL;
        }
        double s = std::sqrt(1.5 * (double)a.n * T / c.ke);
        MD_CUDA(launch(kt.rescale, grid_atoms(), kBlock, a, s));
        return MD_OK;
    }

    int measure(md_measure_t* out) override {
        DevGuard dg(device);
        if (!out) {
            err = "NULL output";
            return MD_EINVAL;
        }
        if (!have_state) {
            err = "md_measure before md_set_state";
            return MD_ESTATE;
        }
        MD_CUDA(launch(kt.finalize, 1, kBlock, a));
        Counters c;
        int r = read_counters(&c);
        if (r) return r;
        std::memset(out, 0, sizeof(*out));
        double V = box[0] * box[1] * box[2];
        out->ke = c.ke;
        out->pe = c.pe;
        out->virial = c.virial;
        out->volume = V;
        out->pressure = (2.0 * c.ke + c.virial) / (3.0 * V);
        out->temperature = 2.0 * c.ke / (3.0 * (double)a.n);
        out->e_tot_per_atom = (c.ke + c.pe) / (double)a.n;
        out->step = c.step;
        out->rebuilds = c.rebuilds;
        out->reorders = c.reorders;
        out->list_entries = c.list_entries;
        out->max_neighbors = c.max_nn;
        out->max_occupancy = c.max_occ;
        out->nbr_capacity = a.cap;
        return MD_OK;
    }

    int get_state(double* pos, double* vel, bool device) override {
        DevGuard dg(this->device);
        if (!pos || !vel) {
            err = "NULL output";
            return MD_EINVAL;
        }
        if (!have_state) {
            err = "md_get_state before md_set_state";
            return MD_ESTATE;
        }
        MD_CUDA(launch(kt.get_state, grid_atoms(), kBlock, a));
        size_t bytes = sizeof(double) * 3 * (size_t)a.n;
        cudaMemcpyKind k = device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        MD_CUDA(cudaMemcpyAsync(pos, a.io_pos, bytes, k, stream));
        MD_CUDA(cudaMemcpyAsync(vel, a.io_vel, bytes, k, stream));
        MD_CUDA(cudaStreamSynchronize(stream));
        return MD_OK;
    }

    int get_forces(double* f) override {
        DevGuard dg(device);
        if (!f) {
            err = "NULL output";
            return MD_EINVAL;
        }
        if (!have_state) {
            err = "md_get_forces before md_set_state";
            return MD_ESTATE;
        }
        double* tmp = a.io_pos;
        MD_CUDA(launch(kt.get_forces, grid_atoms(), kBlock, a, tmp));
        MD_CUDA(cudaMemcpyAsync(f, tmp, sizeof(double) * 3 * (size_t)a.n, cudaMemcpyDeviceToHost, stream));
        MD_CUDA(cudaStreamSynchronize(stream));
        return MD_OK;
    }

    int debug_cells(int32_t* cell) override {
        DevGuard dg(device);
        if (!cell) {
            err = "NULL output";
            return MD_EINVAL;
        }
        if (!have_state) {
            err = "md_debug_cells before md_set_state";
            return MD_ESTATE;
        }
        int* tmp = a.rank;
        MD_CUDA(launch(kt.get_cells, grid_atoms(), kBlock, a, tmp));
        MD_CUDA(cudaMemcpyAsync(cell, tmp, sizeof(int) * (size_t)a.n, cudaMemcpyDeviceToHost, stream));
        MD_CUDA(cudaStreamSynchronize(stream));
        return MD_OK;
    }

    int debug_neighbors(int64_t* count, int64_t* entries, int32_t* pairs, int64_t cap) override {
        DevGuard dg(device);
        if (!count) {
            err = "NULL count";
            return MD_EINVAL;
        }
        if (!have_state) {
            err = "md_debug_neighbors before md_set_state";
            return MD_ESTATE;
        }
        if (prm.cell_list_only) {
            err = "no neighbour list in cell-list-only mode";
            return MD_ESTATE;
        }
        int64_t n = a.n;
        size_t cols = (size_t)((n + 31) / 32) * 32;
        std::vector<int> nn(n), perm(n), nbr(cols * (size_t)a.cap);
        MD_CUDA(cudaMemcpyAsync(nn.data(), a.nn, sizeof(int) * n, cudaMemcpyDeviceToHost, stream));
        MD_CUDA(cudaMemcpyAsync(perm.data(), a.perm, sizeof(int) * n, cudaMemcpyDeviceToHost, stream));
        MD_CUDA(cudaMemcpyAsync(nbr.data(), a.nbr, sizeof(int) * nbr.size(), cudaMemcpyDeviceToHost, stream));
        MD_CUDA(cudaStreamSynchronize(stream));
        int64_t np = 0, ne = 0;
        const int cs = list_stride(a);
        for (int64_t i = 0; i < n; i++) {
            const int* col = nbr.data() + list_base(a, i);
            for (int m = 0; m < nn[i]; m++) {
                int j = col[(size_t)m * cs] & kIndexMask;
                if (j >= n) {
                    err = "neighbour entry out of range";
                    return MD_ECUDA;
                }
                ne++;
                int ui = perm[i], uj = perm[j];
                if (ui < uj) {
                    if (pairs && np < cap) {
                        pairs[2 * np + 0] = ui;
                        pairs[2 * np + 1] = uj;
                    }
                    np++;
                }
            }
        }
        *count = np;
        if (entries) *entries = ne;
        return MD_OK;
    }

    int get_plan(md_plan_t* out) override {
        if (!out) return MD_EINVAL;
        *out = plan;
        out->nbr_capacity = a.cap;
        return MD_OK;
    }

    int set_profiling(int on) override {
        profiling = on != 0;
        return MD_OK;
    }

    int kernel_stats(md_kernel_stats_t* out) override {
        DevGuard dg(device);
        if (!out) return MD_EINVAL;
        Counters c;
        int r = read_counters(&c);
        if (r) return r;
        std::memset(out, 0, sizeof(*out));
        // every rebuild branch that ran launched its kernels
        int per_rebuild = prm.cell_list_only ? 7 : 8;
        int64_t body = prm.use_graphs && !profiling ? (int64_t)c.rebuilds * per_rebuild : 0;
        out->launches = launches + body;
        out->step_kernel_launches = step_launches;
        out->step_kernel_ms = step_ms;
        out->step_kernel_atoms = step_launches * a.n;
        out->step_kernel_bytes = step_bytes;
        out->rebuilds_timed = rebuilds_timed;
        out->rebuild_ms = rebuild_ms;
        return MD_OK;
    }

    int sync() override {
        DevGuard dg(device);
        MD_CUDA(cudaStreamSynchronize(stream));
        Counters c;
        int r = read_counters(&c);
        if (r) return r;
        return check_fatal(c);
    }
};

}  // namespace

namespace md {
__attribute__((visibility("hidden"))) void set_call_error(const char* msg) { g_create_error = msg ? msg : ""; }
}  // namespace md

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

struct md_handle {
    SimBase* sim;
};

extern "C" {

void md_default_params(md_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->precision = MD_PREC_MIXED;
    p->reorder_interval = 100;
    p->cell_list_only = 0;
    p->even_cells = 0;
    p->nbr_capacity = 0;
    p->use_graphs = 1;
    p->device = -1;
    p->shell_bins = 1;
    p->ushift = NAN;
    p->stream = nullptr;
}

int md_plan(const double box[3], int64_t n, double rc, double skin, double dt, const md_params* p,
            md_plan_t* out) {
    std::string why;
    int r = resolve_plan(box, n, rc, skin, dt, p, out, &why);
    if (r) g_create_error = why;
    return r;
}

int md_create(const double box[3], int64_t n, double rc, double skin, double dt, const md_params* p,
              md_handle** out) {
    if (!out) {
        g_create_error = "NULL output handle";
        return MD_EINVAL;
    }
    *out = nullptr;
    md_params d;
    md_default_params(&d);
    const md_params* q = p ? p : &d;
    SimBase* s = nullptr;
    int r;
    if (q->precision == MD_PREC_FP64) {
        auto* sim = new Sim<F64>();
        r = sim->create(box, n, rc, skin, dt, q);
        s = sim;
    } else {
        auto* sim = new Sim<Mixed>();
        r = sim->create(box, n, rc, skin, dt, q);
        s = sim;
    }
    if (r) {
        g_create_error = s->err;
        delete s;
        return r;
    }
    *out = new md_handle{s};
    return MD_OK;
}

#define MD_HANDLE_CHECK(h) \
    if (!(h) || !(h)->sim) return MD_EINVAL

int md_set_state(md_handle* h, const double* pos, const double* vel) {
    MD_HANDLE_CHECK(h);
    return h->sim->set_state(pos, vel, false);
}
int md_set_state_device(md_handle* h, const double* pos, const double* vel) {
    MD_HANDLE_CHECK(h);
    return h->sim->set_state(pos, vel, true);
}
int md_step(md_handle* h, int64_t nsteps) {
    MD_HANDLE_CHECK(h);
    return h->sim->step(nsteps);
}
int md_rescale(md_handle* h, double T) {
    MD_HANDLE_CHECK(h);
    return h->sim->rescale(T);
}
int md_measure(md_handle* h, md_measure_t* out) {
    MD_HANDLE_CHECK(h);
    return h->sim->measure(out);
}
int md_get_state(md_handle* h, double* pos, double* vel) {
    MD_HANDLE_CHECK(h);
    return h->sim->get_state(pos, vel, false);
}
int md_get_state_device(md_handle* h, double* pos, double* vel) {
    MD_HANDLE_CHECK(h);
    return h->sim->get_state(pos, vel, true);
}
int md_get_forces(md_handle* h, double* f) {
    MD_HANDLE_CHECK(h);
    return h->sim->get_forces(f);
}
int md_debug_cells(md_handle* h, int32_t* cell) {
    MD_HANDLE_CHECK(h);
    return h->sim->debug_cells(cell);
}
int md_debug_neighbors(md_handle* h, int64_t* count, int64_t* entries, int32_t* pairs, int64_t capacity) {
    MD_HANDLE_CHECK(h);
    return h->sim->debug_neighbors(count, entries, pairs, capacity);
}
int md_get_plan(md_handle* h, md_plan_t* out) {
    MD_HANDLE_CHECK(h);
    return h->sim->get_plan(out);
}
int md_set_profiling(md_handle* h, int on) {
    MD_HANDLE_CHECK(h);
    return h->sim->set_profiling(on);
}
int md_kernel_stats(md_handle* h, md_kernel_stats_t* out) {
    MD_HANDLE_CHECK(h);
    return h->sim->kernel_stats(out);
}
int md_sync(md_handle* h) {
    MD_HANDLE_CHECK(h);
    return h->sim->sync();
}
void md_destroy(md_handle* h) {
    if (!h) return;
    delete h->sim;
    delete h;
}
const char* md_last_error(const md_handle* h) {
    if (!h || !h->sim) return g_create_error.c_str();
    return h->sim->err.c_str();
}
int md_selftest(int64_t n, int64_t failures[4]) {
    if (n <= 0 || !failures) return MD_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return MD_ENODEV;
    }
    KernelTable<Mixed> kt = make_kernel_table<Mixed>();
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, 4 * sizeof(unsigned long long)) != cudaSuccess) return MD_ENOMEM;
    cudaMemset(d, 0, 4 * sizeof(unsigned long long));
    long long nn = (long long)n;
    void* args[] = {&nn, &d};
    unsigned grid = (unsigned)((n + kBlock - 1) / kBlock);
    cudaError_t e = cudaLaunchKernel(kt.selftest, dim3(grid), dim3(kBlock), args, 0, 0);
    unsigned long long h[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        g_create_error = cudaGetErrorString(e);
        return MD_ECUDA;
    }
    for (int k = 0; k < 4; k++) failures[k] = (int64_t)h[k];
    return MD_OK;
}

const char* md_strerror(int code) {
    switch (code) {
        case MD_OK: return "ok";
        case MD_EINVAL: return "invalid argument";
        case MD_ENOMEM: return "out of memory";
        case MD_ECUDA: return "CUDA error";
        case MD_ESTATE: return "invalid call order";
        case MD_EOVERFLOW: return "neighbour list overflow";
        case MD_EUNSTABLE: return "unstable simulation";
        case MD_ENODEV: return "no CUDA device";
        default: return "unknown error";
    }
}

}  // extern "C"
