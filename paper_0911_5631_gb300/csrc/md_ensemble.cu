// md_ensemble.cu -- host runtime of ensembles (md_ensemble_* in include/md.h).
//
// An ensemble owns one device arena.  Each replica's arrays (the same set a
// single simulation allocates) are carved out of it as one block, so
// admission is a question of arena space and nothing is allocated while
// replicas run.  md_ensemble_run builds a job list (replicas in decreasing
// order of atoms x steps) and launches the per-replica engine k_ensemble
// once: every thread block takes the next job, so large replicas start
// first and small ones fill the gaps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/md.h"
#include "md_common.cuh"
#include "md_host.h"
#include "md_table.h"

namespace {

using namespace md;
using A = Args<Mixed>;

thread_local std::string g_ens_create_error;

constexpr int64_t kAlign = 256;

int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over [0, size) with coalescing of free neighbours.
class Arena {
  public:
    void reset(int64_t size) {
        free_.clear();
        if (size > 0) free_[0] = size;
    }
    int64_t alloc(int64_t bytes) {  // -1 when nothing fits
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                int64_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off, int64_t bytes) {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t largest() const {
        int64_t m = 0;
        for (auto& kv : free_) m = std::max(m, kv.second);
        return m;
    }

  private:
    std::map<int64_t, int64_t> free_;  // offset -> length
};

// Byte layout of one replica's block: every array at a kAlign boundary.
struct Layout {
    int64_t total = 0;
    int64_t take(int64_t bytes) {
        int64_t off = total;
        total += align_up(bytes > 0 ? bytes : 16);
        return off;
    }
};

int replica_plan(const md_replica_desc* d, md_plan_t* plan, md_params* prm, std::string* why) {
    if (!d) {
        if (why) *why = "NULL replica description";
        return MD_EINVAL;
    }
    for (int k = 0; k < 4; k++)
        if (d->reserved[k] != 0) {
            if (why) *why = "reserved fields of md_replica_desc must be zero";
            return MD_EINVAL;
        }
    md_default_params(prm);
    prm->precision = MD_PREC_MIXED;
    prm->reorder_interval = d->reorder_interval;
    prm->nbr_capacity = d->nbr_capacity;
    prm->ushift = d->ushift;
    if (d->skin <= 0.0) {
        if (why) *why = "ensemble replicas need skin > 0 (neighbour-list form)";
        return MD_EINVAL;
    }
    return resolve_plan(d->box, d->n, d->rc, d->skin, d->dt, prm, plan, why);
}

// Lays out the arrays of one replica at base (device address; 0 for sizing).
int64_t lay_out(A& a, const md_plan_t& plan, char* base) {
    Layout L;
    const int64_t n = a.n, nc = plan.n_cells;
    auto at = [&](auto*& p, int64_t count) {
        using T = std::remove_reference_t<decltype(*p)>;
        int64_t off = L.take(count * (int64_t)sizeof(T));
        p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    };
    at(a.cell, n); at(a.perm, n); at(a.rank, n);
    at(a.pbx, n); at(a.pby, n); at(a.pbz, n);
    at(a.ox, n); at(a.oy, n); at(a.oz, n);
    at(a.vx, n); at(a.vy, n); at(a.vz, n);
    at(a.fx, n); at(a.fy, n); at(a.fz, n);
    at(a.pA, pair_slots(n)); at(a.pB, pair_slots(n)); at(a.cand, n);
    at(a.s_cell, n); at(a.s_perm, n);
    at(a.s_pbx, n); at(a.s_pby, n); at(a.s_pbz, n);
    at(a.s_ox, n); at(a.s_oy, n); at(a.s_oz, n);
    at(a.s_vx, n); at(a.s_vy, n); at(a.s_vz, n);
    at(a.count, nc); at(a.cell_start, nc + 1);
    at(a.order, n); at(a.tile_sum, 1);
    at(a.nn, n); at(a.lim, (kShellBins - 1) * n);
    at(a.nbr, (n + 31) / 32 * 32 * (int64_t)(a.cap > 0 ? a.cap : 1));
    {  // per-chunk (32 atoms) and per-group (32 chunks) energy partials
        const int64_t nch = (n + 31) / 32;
        at(a.part, 3 * (nch + (nch + 31) / 32));
    }
    at(a.ctr, 1);
    at(a.io_pos, 3 * n); at(a.io_vel, 3 * n);
    return L.total;
}

struct Replica {
    bool used = false;
    md_replica_desc d{};
    md_plan_t plan{};
    A a{};
    int64_t off = -1, bytes = 0;
    bool pending_init = false;
    bool ever_run = false;
    int last_run = -1;     // index of the last run that included it
    int last_slot = -1;    // its job slot in that run
};

}  // namespace

constexpr int kRunEvents = 8;  // events of the most recent runs, reused in a ring

struct md_ensemble {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // Host-side calls on one replica (add, measure, status, get_state) run
    // their copies on a stream of their own after an event of the replica's
    // last run, so that they overlap the runs queued after it.
    cudaStream_t xs = nullptr;
    cudaEvent_t run_ev[kRunEvents] = {};
    char* arena = nullptr;
    int64_t arena_bytes = 0;
    Arena alloc;
    A* d_args = nullptr;
    int max_replicas = 0;
    EnsJob* d_jobs = nullptr;
    int jobs_cap = 0;
    int* d_next = nullptr;      // {queue[0], queue[1], njobs, nteam} of a launch
    // Launches are replayed from CUDA graphs, one per launch shape (and job
    // buffer): each run copies the job list and the header, then launches
    // the graph.
    struct Launch {
        int block = 0, grid = 0, cluster = 0;
        EnsJob* jobs = nullptr;
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<Launch> graphs;
    EnsJob* h_jobs = nullptr;  // pinned copy of the last run's jobs
    int h_jobs_cap = 0;
    int last_njobs = 0;
    int runs = 0;
    bool jobs_valid = false;   // h_jobs holds the finished last run
    unsigned long long launch_t0 = 0;
    std::vector<Replica> reps;
    KernelTable<Mixed> kt{};
    int block = 256, grid = 0;
    int cluster = 8;            // blocks per team for big replicas (1: no teams)
    int64_t team_atoms = 8192;  // replicas with at least this many atoms get a team
    std::string err;
};

namespace {

#define ENS_CUDA(call)                                                               \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            e->err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
            return e_ == cudaErrorMemoryAllocation ? MD_ENOMEM : MD_ECUDA;           \
        }                                                                            \
    } while (0)

struct EnsDev {
    int prev = -1;
    bool changed = false;
    explicit EnsDev(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) changed = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~EnsDev() {
        if (changed && prev >= 0) cudaSetDevice(prev);
    }
};

int bad_id(md_ensemble* e, int32_t id) {
    if (id < 0 || id >= (int)e->reps.size() || !e->reps[id].used) {
        e->err = "unknown replica id";
        return MD_EINVAL;
    }
    return MD_OK;
}

int ensure_jobs(md_ensemble* e, int n) {
    if (n <= e->jobs_cap) return MD_OK;
    ENS_CUDA(cudaStreamSynchronize(e->stream));  // the old array may still be in use
    if (e->d_jobs) cudaFree(e->d_jobs);
    e->d_jobs = nullptr;
    e->jobs_cap = 0;
    int cap = std::max(n, 64);
    ENS_CUDA(cudaMalloc(&e->d_jobs, sizeof(EnsJob) * cap));
    e->jobs_cap = cap;
    return MD_OK;
}

int ensure_host_jobs(md_ensemble* e, int n) {
    if (n <= e->h_jobs_cap) return MD_OK;
    if (e->h_jobs) cudaFreeHost(e->h_jobs);
    e->h_jobs = nullptr;
    e->h_jobs_cap = 0;
    int cap = std::max(n, 64);
    ENS_CUDA(cudaMallocHost(&e->h_jobs, sizeof(EnsJob) * cap));
    e->h_jobs_cap = cap;
    return MD_OK;
}

// Copies the finished last run's jobs to the host (once per run).
int fetch_jobs(md_ensemble* e) {
    if (e->jobs_valid || e->last_njobs == 0) return MD_OK;
    int r = ensure_host_jobs(e, e->last_njobs);
    if (r) return r;
    ENS_CUDA(cudaMemcpyAsync(e->h_jobs, e->d_jobs, sizeof(EnsJob) * e->last_njobs, cudaMemcpyDeviceToHost, e->stream));
    ENS_CUDA(cudaStreamSynchronize(e->stream));
    e->jobs_valid = true;
    return MD_OK;
}

// The event recorded after run r (1-based).  Once kRunEvents later runs
// have been queued it holds a later run, whose completion implies run r's.
cudaEvent_t run_event(md_ensemble* e, int r) { return e->run_ev[(r - 1) % kRunEvents]; }

// Orders the transfer stream after the last run that included the replica.
int after_last_run(md_ensemble* e, const Replica& rp) {
    if (rp.last_run >= 1) ENS_CUDA(cudaStreamWaitEvent(e->xs, run_event(e, rp.last_run), 0));
    return MD_OK;
}

int read_counters(md_ensemble* e, const Replica& rp, Counters* c) {
    int r = after_last_run(e, rp);
    if (r) return r;
    ENS_CUDA(cudaMemcpyAsync(c, rp.a.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, e->xs));
    ENS_CUDA(cudaStreamSynchronize(e->xs));
    return MD_OK;
}

int launch_run(md_ensemble* e, const std::vector<EnsJob>& jobs, int nteam, int block, int grid, int cluster) {
    int r = ensure_jobs(e, (int)jobs.size());
    if (r) return r;
    // from pageable memory: the call has read `jobs` when it returns
    ENS_CUDA(cudaMemcpyAsync(e->d_jobs, jobs.data(), sizeof(EnsJob) * jobs.size(), cudaMemcpyHostToDevice, e->stream));
    int nj = (int)jobs.size();
    if (nteam == 0) cluster = 1;
    const int hdr[4] = {0, 0, nj, nteam};  // pageable too: read when the call returns
    ENS_CUDA(cudaMemcpyAsync(e->d_next, hdr, sizeof(hdr), cudaMemcpyHostToDevice, e->stream));
    size_t smem = (size_t)block * kEnsSmemInts * sizeof(int);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = e->stream;
    if (cluster > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    int g = grid;
    if (g <= 0) {
        if (cluster > 1) {
            int nclusters = 0;
            cfg.gridDim = dim3(cluster);
            ENS_CUDA(cudaOccupancyMaxActiveClusters(&nclusters, (const void*)e->kt.ensemble, &cfg));
            g = std::max(1, nclusters) * cluster;
        } else {
            int per_sm = 0, sms = 0;
            ENS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)e->kt.ensemble, block, smem));
            ENS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device));
            g = std::max(1, per_sm) * sms;
        }
    }
    if (cluster > 1) g = (g + cluster - 1) / cluster * cluster;
    cfg.gridDim = dim3(g);
    // blocks without a job leave at their first queue read, so one graph
    // per shape serves every job list
    md_ensemble::Launch* lg = nullptr;
    for (auto& x : e->graphs)
        if (x.block == block && x.grid == g && x.cluster == cluster && x.jobs == e->d_jobs) lg = &x;
    if (!lg) {
        void* args[] = {(void*)&e->d_args, (void*)&e->d_jobs, (void*)&e->d_next};
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        ENS_CUDA(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t lc = cudaLaunchKernelExC(&cfg, e->kt.ensemble, args);
        cudaError_t ec = cudaStreamEndCapture(e->stream, &graph);
        if (lc != cudaSuccess || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            e->err = std::string("capturing the ensemble launch: ") + cudaGetErrorString(lc != cudaSuccess ? lc : ec);
            return MD_ECUDA;
        }
        cudaError_t ic = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        ENS_CUDA(ic);
        e->graphs.push_back({block, g, cluster, e->d_jobs, exec});
        lg = &e->graphs.back();
    }
    ENS_CUDA(cudaGraphLaunch(lg->exec, e->stream));
    e->last_njobs = nj;
    e->jobs_valid = false;
    e->runs++;
    ENS_CUDA(cudaEventRecord(run_event(e, e->runs), e->stream));
    return MD_OK;
}

int make_jobs(md_ensemble* e, int32_t count, const int32_t* ids, const int64_t* nsteps, std::vector<EnsJob>* jobs,
              int cluster, int* nteam) {
    if (count < 0 || (count > 0 && (!ids || !nsteps))) {
        e->err = "bad id list";
        return MD_EINVAL;
    }
    std::vector<char> seen(e->reps.size(), 0);
    jobs->clear();
    for (int k = 0; k < count; k++) {
        int r = bad_id(e, ids[k]);
        if (r) return r;
        if (seen[ids[k]]) {
            e->err = "a replica id appears twice in one run";
            return MD_EINVAL;
        }
        seen[ids[k]] = 1;
        if (nsteps[k] < 0) {
            e->err = "negative step count";
            return MD_EINVAL;
        }
        EnsJob j{};
        j.rep = ids[k];
        j.init = e->reps[ids[k]].pending_init ? 1 : 0;
        j.nsteps = nsteps[k];
        jobs->push_back(j);
    }
    // replicas big enough for a team first, then the rest; largest work
    // first within each list, so that blocks taking small jobs later fill
    // the gaps
    auto team = [&](const EnsJob& x) { return cluster > 1 && e->reps[x.rep].a.n >= e->team_atoms; };
    std::stable_sort(jobs->begin(), jobs->end(), [&](const EnsJob& x, const EnsJob& y) {
        if (team(x) != team(y)) return team(x);
        double wx = (double)e->reps[x.rep].a.n * (double)(x.nsteps + x.init);
        double wy = (double)e->reps[y.rep].a.n * (double)(y.nsteps + y.init);
        return wx > wy;
    });
    *nteam = 0;
    for (auto& j : *jobs) *nteam += team(j) ? 1 : 0;
    return MD_OK;
}

int run_jobs(md_ensemble* e, std::vector<EnsJob>& jobs, int nteam, int block, int grid, int cluster) {
    if (jobs.empty()) return MD_OK;
    int r = launch_run(e, jobs, nteam, block, grid, cluster);
    if (r) return r;
    for (size_t k = 0; k < jobs.size(); k++) {
        Replica& rp = e->reps[jobs[k].rep];
        rp.pending_init = false;
        rp.ever_run = true;
        rp.last_run = e->runs;
        rp.last_slot = (int)k;
    }
    return MD_OK;
}

}  // namespace

extern "C" {

int md_ensemble_create(int64_t arena_bytes, int32_t max_replicas, int32_t device, void* stream, md_ensemble** out) {
    g_ens_create_error.clear();
    if (!out) {
        g_ens_create_error = "NULL output";
        return MD_EINVAL;
    }
    *out = nullptr;
    if (arena_bytes <= 0 || max_replicas <= 0) {
        g_ens_create_error = "arena_bytes and max_replicas must be positive";
        return MD_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        g_ens_create_error = "no CUDA device";
        return MD_ENODEV;
    }
    if (device >= ndev) {
        g_ens_create_error = "device ordinal out of range";
        return MD_EINVAL;
    }
    md_ensemble* e = new md_ensemble();
    if (device >= 0) e->device = device;
    else cudaGetDevice(&e->device);
    EnsDev dg(e->device);
    auto fail = [&](int code) {
        g_ens_create_error = e->err;
        md_ensemble_destroy(e);
        return code;
    };
    e->kt = make_kernel_table<Mixed>();
    if (cudaStreamCreateWithFlags(&e->xs, cudaStreamNonBlocking) != cudaSuccess) {
        e->err = "cudaStreamCreateWithFlags failed";
        return fail(MD_ECUDA);
    }
    for (auto& ev : e->run_ev)
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            e->err = "cudaEventCreate failed";
            return fail(MD_ECUDA);
        }
    if (stream) {
        e->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) {
            e->err = "cudaStreamCreateWithFlags failed";
            return fail(MD_ECUDA);
        }
        e->own_stream = true;
    }
    if (cudaMalloc(&e->arena, (size_t)arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        e->err = "cannot allocate the arena";
        return fail(MD_ENOMEM);
    }
    e->arena_bytes = arena_bytes;
    e->alloc.reset(arena_bytes);
    if (cudaMalloc(&e->d_args, sizeof(A) * (size_t)max_replicas) != cudaSuccess ||
        cudaMalloc(&e->d_next, 4 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        e->err = "cannot allocate the replica table";
        return fail(MD_ENOMEM);
    }
    e->max_replicas = max_replicas;
    // the engine's staged rows and build staging need more than the default
    // 48 KB of dynamic shared memory at 1024 threads
    int smax = 1024 * kEnsSmemInts * (int)sizeof(int);
    if (cudaFuncSetAttribute(e->kt.ensemble, cudaFuncAttributeMaxDynamicSharedMemorySize, smax) != cudaSuccess) {
        cudaGetLastError();
        e->err = "cudaFuncSetAttribute failed";
        return fail(MD_ECUDA);
    }
    *out = e;
    return MD_OK;
}

int64_t md_ensemble_replica_bytes(const md_replica_desc* d) {
    md_plan_t plan;
    md_params prm;
    if (replica_plan(d, &plan, &prm, nullptr)) return 0;
    A a{};
    a.n = d->n;
    a.cap = plan.nbr_capacity;
    return lay_out(a, plan, nullptr);
}

int64_t md_ensemble_free_bytes(const md_ensemble* e) { return e ? e->alloc.largest() : 0; }

int md_ensemble_add(md_ensemble* e, const md_replica_desc* d, const double* pos, const double* vel, int32_t* id) {
    if (!e) return MD_EINVAL;
    EnsDev dg(e->device);
    if (!id || !pos || !vel) {
        e->err = "NULL argument";
        return MD_EINVAL;
    }
    md_plan_t plan;
    md_params prm;
    int r = replica_plan(d, &plan, &prm, &e->err);
    if (r) return r;
    int slot = -1;
    for (int k = 0; k < (int)e->reps.size(); k++)
        if (!e->reps[k].used) {
            slot = k;
            break;
        }
    if (slot < 0) {
        if ((int)e->reps.size() >= e->max_replicas) {
            e->err = "replica table full";
            return MD_ENOMEM;
        }
        e->reps.emplace_back();
        slot = (int)e->reps.size() - 1;
    }
    Replica rp;
    rp.d = *d;
    rp.plan = plan;
    fill_args_scalars(rp.a, plan, d->box, d->n, d->rc, d->skin, d->dt, 0, d->reorder_interval);
    rp.bytes = lay_out(rp.a, plan, nullptr);
    rp.off = e->alloc.alloc(rp.bytes);
    if (rp.off < 0) {
        if (slot == (int)e->reps.size() - 1 && !e->reps[slot].used) e->reps.pop_back();
        e->err = "arena full";
        return MD_ENOMEM;
    }
    lay_out(rp.a, plan, e->arena + rp.off);
    rp.used = true;
    rp.pending_init = true;
    size_t bytes = sizeof(double) * 3 * (size_t)d->n;
    auto undo = [&](int code) {
        e->alloc.release(rp.off, rp.bytes);
        if (slot == (int)e->reps.size() - 1) e->reps.pop_back();
        return code;
    };
    // On the transfer stream: the arena space and the table slot belong to
    // no queued run (a removed replica's last run had finished), so the
    // copies may overlap the runs in flight.
    cudaError_t c1 = cudaMemcpyAsync(rp.a.io_pos, pos, bytes, cudaMemcpyHostToDevice, e->xs);
    cudaError_t c2 = cudaMemcpyAsync(rp.a.io_vel, vel, bytes, cudaMemcpyHostToDevice, e->xs);
    cudaError_t c3 = cudaMemsetAsync(rp.a.count, 0, sizeof(int) * (size_t)rp.a.ncells, e->xs);
    cudaError_t c4 = cudaMemsetAsync(rp.a.nn, 0, sizeof(int) * (size_t)rp.a.n, e->xs);
    cudaError_t c5 = cudaMemsetAsync(rp.a.ctr, 0, sizeof(Counters), e->xs);
    cudaError_t c6 = cudaMemcpyAsync(e->d_args + slot, &rp.a, sizeof(A), cudaMemcpyHostToDevice, e->xs);
    if (c1 || c2 || c3 || c4 || c5 || c6) {
        e->err = "copying the replica's state failed";
        return undo(MD_ECUDA);
    }
    // the host copy of the arguments (pageable) must outlive the copy, and
    // the next run must see the state: finish them before returning
    if (cudaStreamSynchronize(e->xs) != cudaSuccess) {
        e->err = "cudaStreamSynchronize failed";
        return undo(MD_ECUDA);
    }
    e->reps[slot] = rp;
    *id = slot;
    return MD_OK;
}

int md_ensemble_remove(md_ensemble* e, int32_t id) {
    if (!e) return MD_EINVAL;
    int r = bad_id(e, id);
    if (r) return r;
    EnsDev dg(e->device);
    Replica& rp = e->reps[id];
    // its memory is free once its last run has finished (later runs do
    // not touch it)
    if (rp.last_run >= 1) ENS_CUDA(cudaEventSynchronize(run_event(e, rp.last_run)));
    e->alloc.release(rp.off, rp.bytes);
    rp = Replica();
    return MD_OK;
}

int md_ensemble_run(md_ensemble* e, int32_t count, const int32_t* ids, const int64_t* nsteps) {
    if (!e) return MD_EINVAL;
    EnsDev dg(e->device);
    std::vector<EnsJob> jobs;
    int nteam = 0;
    int r = make_jobs(e, count, ids, nsteps, &jobs, e->cluster, &nteam);
    if (r) return r;
    return run_jobs(e, jobs, nteam, e->block, e->grid, e->cluster);
}

int md_ensemble_sync(md_ensemble* e) {
    if (!e) return MD_EINVAL;
    EnsDev dg(e->device);
    ENS_CUDA(cudaStreamSynchronize(e->stream));
    return MD_OK;
}

int md_ensemble_wait(md_ensemble* e, int32_t in_flight) {
    if (!e) return MD_EINVAL;
    if (in_flight < 0 || in_flight >= kRunEvents) {
        e->err = "in_flight must be in 0..7";
        return MD_EINVAL;
    }
    EnsDev dg(e->device);
    if (in_flight == 0) {
        ENS_CUDA(cudaStreamSynchronize(e->stream));
        return MD_OK;
    }
    const int r = e->runs - in_flight;
    if (r >= 1) ENS_CUDA(cudaEventSynchronize(run_event(e, r)));
    return MD_OK;
}

int md_ensemble_status(md_ensemble* e, int32_t id) {
    if (!e) return MD_EINVAL;
    int r = bad_id(e, id);
    if (r) return r;
    EnsDev dg(e->device);
    Counters c;
    r = read_counters(e, e->reps[id], &c);
    if (r) return r;
    if (c.error & kErrOverflow) {
        e->err = "neighbour capacity exceeded (raise nbr_capacity)";
        return MD_EOVERFLOW;
    }
    if (c.error & (kErrUnstable | kErrClose)) {
        e->err = (c.error & kErrClose) ? "two atoms came closer than the fixed-point force range allows"
                                       : "non-finite coordinate or velocity";
        return MD_EUNSTABLE;
    }
    return MD_OK;
}

int md_ensemble_measure(md_ensemble* e, int32_t id, md_measure_t* out) {
    if (!e) return MD_EINVAL;
    int r = bad_id(e, id);
    if (r) return r;
    if (!out) {
        e->err = "NULL output";
        return MD_EINVAL;
    }
    Replica& rp = e->reps[id];
    if (!rp.ever_run) {
        e->err = "replica not loaded yet (run it first)";
        return MD_ESTATE;
    }
    EnsDev dg(e->device);
    Counters c;
    r = read_counters(e, rp, &c);
    if (r) return r;
    std::memset(out, 0, sizeof(*out));
    const double V = rp.d.box[0] * rp.d.box[1] * rp.d.box[2];
    out->ke = c.ke;
    out->pe = c.pe;
    out->virial = c.virial;
    out->volume = V;
    out->pressure = (2.0 * c.ke + c.virial) / (3.0 * V);
    out->temperature = 2.0 * c.ke / (3.0 * (double)rp.a.n);
    out->e_tot_per_atom = (c.ke + c.pe) / (double)rp.a.n;
    out->step = c.step;
    out->rebuilds = c.rebuilds;
    out->reorders = c.reorders;
    out->list_entries = c.list_entries;
    out->max_neighbors = c.max_nn;
    out->max_occupancy = c.max_occ;
    out->nbr_capacity = rp.a.cap;
    return MD_OK;
}

int md_ensemble_get_state(md_ensemble* e, int32_t id, double* pos, double* vel) {
    if (!e) return MD_EINVAL;
    int r = bad_id(e, id);
    if (r) return r;
    if (!pos || !vel) {
        e->err = "NULL output";
        return MD_EINVAL;
    }
    Replica& rp = e->reps[id];
    if (!rp.ever_run) {
        e->err = "replica not loaded yet (run it first)";
        return MD_ESTATE;
    }
    EnsDev dg(e->device);
    r = after_last_run(e, rp);
    if (r) return r;
    void* args[] = {(void*)&rp.a};
    unsigned grid = (unsigned)((rp.a.n + kBlock - 1) / kBlock);
    ENS_CUDA(cudaLaunchKernel(e->kt.get_state, dim3(grid), dim3(kBlock), args, 0, e->xs));
    size_t bytes = sizeof(double) * 3 * (size_t)rp.a.n;
    ENS_CUDA(cudaMemcpyAsync(pos, rp.a.io_pos, bytes, cudaMemcpyDeviceToHost, e->xs));
    ENS_CUDA(cudaMemcpyAsync(vel, rp.a.io_vel, bytes, cudaMemcpyDeviceToHost, e->xs));
    ENS_CUDA(cudaStreamSynchronize(e->xs));
    return MD_OK;
}

int md_ensemble_times(md_ensemble* e, int32_t count, const int32_t* ids, double* start_ms, double* end_ms) {
    if (!e) return MD_EINVAL;
    if (count < 0 || (count > 0 && (!ids || !start_ms || !end_ms))) {
        e->err = "NULL argument";
        return MD_EINVAL;
    }
    EnsDev dg(e->device);
    int r = fetch_jobs(e);
    if (r) return r;
    unsigned long long t0 = ~0ull;
    for (int k = 0; k < e->last_njobs; k++) t0 = std::min(t0, e->h_jobs[k].t_start);
    for (int k = 0; k < count; k++) {
        r = bad_id(e, ids[k]);
        if (r) return r;
        const Replica& rp = e->reps[ids[k]];
        start_ms[k] = end_ms[k] = -1.0;
        if (rp.last_run == e->runs && rp.last_slot >= 0 && rp.last_slot < e->last_njobs) {
            const EnsJob& j = e->h_jobs[rp.last_slot];
            start_ms[k] = (double)(j.t_start - t0) * 1e-6;
            end_ms[k] = (double)(j.t_end - t0) * 1e-6;
        }
    }
    return MD_OK;
}

int md_ensemble_set_shape(md_ensemble* e, int32_t block, int32_t grid, int32_t cluster, int64_t team_atoms) {
    if (!e) return MD_EINVAL;
    if (block == 0) block = 256;
    if (cluster == 0) cluster = 8;
    if (team_atoms == 0) team_atoms = 8192;
    if (block < 64 || block > 1024 || block % 32 != 0 || grid < 0 || cluster < 1 || cluster > 8 ||
        team_atoms < 0) {
        e->err = "block must be a multiple of 32 in 64..1024, grid >= 0, cluster in 1..8, team_atoms >= 0";
        return MD_EINVAL;
    }
    e->block = block;
    e->grid = grid;
    e->cluster = cluster;
    e->team_atoms = team_atoms;
    return MD_OK;
}

int md_ensemble_autotune(md_ensemble* e, int32_t count, const int32_t* ids, int64_t probe_steps, int32_t* block,
                         int32_t* cluster) {
    if (!e) return MD_EINVAL;
    if (probe_steps <= 0) {
        e->err = "probe_steps must be positive";
        return MD_EINVAL;
    }
    EnsDev dg(e->device);
    int nteam = 0;
    {  // load pending replicas first, so that every candidate times the same work
        std::vector<int64_t> zero(count, 0);
        std::vector<EnsJob> jobs;
        int r0 = make_jobs(e, count, ids, zero.data(), &jobs, e->cluster, &nteam);
        if (r0) return r0;
        bool pending = false;
        for (auto& j : jobs) pending |= j.init != 0;
        if (pending) {
            r0 = run_jobs(e, jobs, nteam, e->block, e->grid, e->cluster);
            if (r0) return r0;
        }
    }
    std::vector<int64_t> steps(count, probe_steps);
    // candidate shapes: (threads per block, blocks per team, atoms from which
    // a replica gets a team)
    const int cands[][3] = {{256, 1, 0}, {1024, 1, 0}, {1024, 2, 8192}, {1024, 4, 8192},
                            {1024, 4, 16384}, {1024, 8, 16384}};
    const int64_t saved_team = e->team_atoms;
    float best = -1.f;
    int best_b = e->block, best_c = e->cluster;
    int64_t best_t = e->team_atoms;
    cudaEvent_t t0, t1;
    ENS_CUDA(cudaEventCreate(&t0));
    ENS_CUDA(cudaEventCreate(&t1));
    int r = MD_OK;
    for (auto& c : cands) {
        std::vector<EnsJob> jobs;
        e->team_atoms = c[2] > 0 ? c[2] : saved_team;
        r = make_jobs(e, count, ids, steps.data(), &jobs, c[1], &nteam);
        if (r) break;
        if (cudaEventRecord(t0, e->stream) != cudaSuccess) { r = MD_ECUDA; break; }
        r = run_jobs(e, jobs, nteam, c[0], 0, c[1]);
        if (r) break;
        if (cudaEventRecord(t1, e->stream) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess) {
            r = MD_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (best < 0.f || ms < best) {
            best = ms;
            best_b = c[0];
            best_c = c[1];
            best_t = e->team_atoms;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (r) {
        if (e->err.empty()) e->err = "autotune launch failed";
        return r;
    }
    e->block = best_b;
    e->grid = 0;
    e->cluster = best_c;
    e->team_atoms = r ? saved_team : best_t;
    if (block) *block = best_b;
    if (cluster) *cluster = best_c;
    return MD_OK;
}

void md_ensemble_destroy(md_ensemble* e) {
    if (!e) return;
    EnsDev dg(e->device);
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->xs) {
        cudaStreamSynchronize(e->xs);
        cudaStreamDestroy(e->xs);
    }
    for (auto& ev : e->run_ev)
        if (ev) cudaEventDestroy(ev);
    if (e->arena) cudaFree(e->arena);
    if (e->d_args) cudaFree(e->d_args);
    if (e->d_jobs) cudaFree(e->d_jobs);
    if (e->d_next) cudaFree(e->d_next);
    for (auto& x : e->graphs)
        if (x.exec) cudaGraphExecDestroy(x.exec);
    if (e->h_jobs) cudaFreeHost(e->h_jobs);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

const char* md_ensemble_last_error(const md_ensemble* e) {
    if (!e) return g_ens_create_error.c_str();
    return e->err.c_str();
}

}  // extern "C"
