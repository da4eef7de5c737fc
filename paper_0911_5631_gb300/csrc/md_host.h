// md_host.h -- host-side helpers shared by the single-simulation runtime
// (md_api.cu) and the ensemble runtime (md_ensemble.cu).  Internal.
#pragma once

#include <cmath>
#include <cstring>
#include <string>

#include "../../include/md.h"
#include "md_common.cuh"

namespace md {

// Geometry and sizes of one simulation (Sec. 3.1: G_d = floor(L_d / r_n),
// optionally even; cell width w_d = L_d / G_d; neighbour capacity from the
// density unless given), with the argument checks of md_plan.
inline int resolve_plan(const double box[3], int64_t n, double rc, double skin, double dt, const md_params* p,
                        md_plan_t* out, std::string* why) {
    md_params d;
    md_default_params(&d);
    if (!p) p = &d;
    auto fail = [&](const char* m) {
        if (why) *why = m;
        return MD_EINVAL;
    };
    if (!box || !out) return fail("NULL argument");
    if (n <= 0) return fail("n must be positive");
    if (n >= md::kMaxAtoms) return fail("n must be below 2^26 (neighbour entries carry a 6-bit cell code)");
    if (!(rc > 0.0) || !std::isfinite(rc)) return fail("rc must be positive and finite");
    if (!(skin >= 0.0) || !std::isfinite(skin)) return fail("skin must be non-negative and finite");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail("dt must be positive and finite");
    if (p->precision != MD_PREC_MIXED && p->precision != MD_PREC_FP64) return fail("unknown precision");
    if (p->cell_list_only && skin != 0.0) return fail("cell_list_only requires skin == 0");
    if (p->reorder_interval < 0) return fail("reorder_interval must be >= 0");
    if (p->nbr_capacity < 0) return fail("nbr_capacity must be >= 0");
    if (p->build_kernel < MD_BUILD_AUTO || p->build_kernel > MD_BUILD_WARP) return fail("unknown build_kernel");
    if (p->variant != 0) {
        const int v = p->variant;
        if (v != MD_VARIANT_PLAIN_LOADS && v != MD_VARIANT_LIST_ROWS && v != MD_VARIANT_BLOCK64 &&
            v != MD_VARIANT_BLOCK256)
            return fail("variant must be 0 or a single MD_VARIANT_* flag");
        if (p->precision != MD_PREC_MIXED || p->cell_list_only)
            return fail("kernel variants exist for the mixed form with a neighbour list only");
    }
    std::memset(out, 0, sizeof(*out));
    double rn = rc + skin;
    int64_t nc = 1;
    for (int k = 0; k < 3; k++) {
        if (!(box[k] > 0.0) || !std::isfinite(box[k])) return fail("box edges must be positive and finite");
        double g = std::floor(box[k] / rn);
        if (g > 1e6) return fail("too many cells along one edge");
        int G = (int)g;
        if (p->even_cells) G -= G % 2;
        if (G < 3) return fail("box edge below 3 r_n: the 27-cell neighbourhood would alias");
        if (G > 1023) return fail("more than 1023 cells along one edge");
        out->G[k] = G;
        out->w[k] = box[k] / G;
        nc *= G;
    }
    if (nc > (int64_t)1 << 30) return fail("too many cells");
    out->n_cells = nc;
    out->rn = rn;
    if (std::isnan(p->ushift)) {
        double wca = std::pow(2.0, 1.0 / 6.0);
        out->ushift = std::fabs(rc - wca) <= 1e-12 * rc ? 1.0 : 0.0;
    } else {
        out->ushift = p->ushift;
    }
    int cap = 0;
    if (!p->cell_list_only) {
        if (p->nbr_capacity > 0) {
            cap = p->nbr_capacity;
        } else {
            double rho = (double)n / (box[0] * box[1] * box[2]);
            double nbar = 4.0 / 3.0 * M_PI * rn * rn * rn * rho;
            cap = (int)std::ceil(nbar + 6.0 * std::sqrt(nbar) + 8.0);
        }
        cap = (cap + 3) & ~3;  // a multiple of 4 (the step kernel reads its staged rows four at a time)
        if (cap < 8) cap = 8;
        int cap_max = p->precision == MD_PREC_MIXED ? md::kMaxCapMixed : 4096;
        if (cap > cap_max) cap = cap_max;
    }
    out->nbr_capacity = cap;
    // device bytes: see Sim::allocate
    int64_t nb = (n + kBlock - 1) / kBlock;
    int64_t real_b = p->precision == MD_PREC_FP64 ? 8 : 4;
    int64_t pos4_b = p->precision == MD_PREC_FP64 ? 32 : 16;
    int64_t per_atom = 3 * 4 /*cell perm rank*/ + 3 * real_b /*pb*/ + 24 /*o*/ + 3 * real_b /*v*/ +
                       3 * real_b /*f*/ + 2 * pos4_b /*pA pB*/ + 16 /*cand*/ + 8 + 3 * real_b + 24 +
                       3 * real_b /*scratch*/ +
                       4 /*order*/ + 4 /*nn*/ + (kShellBins - 1) /*lim*/ + 48 /*io*/;
    int64_t ncol = (n + 31) / 32 * 32;
    out->device_bytes = per_atom * n + 2 * pos4_b * (pair_slots(n) - n) /*pair buffers padded*/ + ncol * cap * 4 +
                        (2 * nc + 1) * 4 + ((nc + kScanTile - 1) / kScanTile) * 4 + 3 * nb * 8 +
                        (int64_t)sizeof(Counters) + kD2Buckets * 32 * 4;
    return MD_OK;
}

// The neighbour-list build a handle uses.  The warp-cooperative build runs
// only when asked for: measured at the 1M-atom workload it takes about twice
// as long as the thread-per-atom build (its per-cell setup and ballot
// compaction are spread over only about three atoms per cell).
inline bool use_warp_build(const md_params& p) { return p.build_kernel == MD_BUILD_WARP; }

// Whether the thread-per-atom build writes entries as it finds them rather
// than staging them for the shell-bin sort: when the expected number of
// entries per atom (the density times the r_n sphere) exceeds the stage
// depth, most atoms would overflow the stage and be scanned twice.  (Below
// it, the few atoms that overflow are scanned twice and keep the shell-bin
// savings of the rest.)
inline bool use_direct_build(const double box[3], int64_t n, double rn) {
    const double nbar = 4.0 / 3.0 * M_PI * rn * rn * rn * (double)n / (box[0] * box[1] * box[2]);
    return nbar > kBuildStage;
}

// Scalar members of Args from a plan.
template <class P>
void fill_args_scalars(Args<P>& a, const md_plan_t& plan, const double box[3], int64_t n, double rc, double skin,
                       double dt, int cell_list_only, int reorder_interval, int shell_bins = 1) {
    a.n = n;
    a.jmask = (unsigned)(pair_slots(n) - 1);
    a.cap = plan.nbr_capacity;
    a.ncells = (int)plan.n_cells;
    for (int k = 0; k < 3; k++) {
        a.G[k] = plan.G[k];
        a.L[k] = box[k];
        a.hL[k] = 0.5 * box[k];
        a.invL[k] = 1.0 / box[k];
        a.invW[k] = (double)plan.G[k] / box[k];
        a.w[k] = plan.w[k];
        a.hw[k] = 0.5 * plan.w[k];
        a.hwf_in[k] = (float)(0.5 * plan.w[k] * (1.0 - 1e-6));
        a.hw_in[k] = 0.5 * plan.w[k] * (1.0 - 1e-9);
        a.wf[k] = (float)plan.w[k];
    }
    a.ntiles = (int)((plan.n_cells + kScanTile - 1) / kScanTile);
    a.nblocks = (int)((n + kBlock - 1) / kBlock);
    a.cell_list_only = cell_list_only;
    a.reorder_interval = reorder_interval;
    a.shell_bins = shell_bins != 0;
    a.list_rows = 0;
    a.dt = dt;
    a.h = 0.5 * dt;
    a.dtf = (float)dt;
    a.hf = (float)(0.5 * dt);
    a.rc2 = rc * rc;
    a.rc2f = (float)a.rc2;
    double rn = rc + skin;
    a.rn2 = rn * rn;
    // FP32 pre-filter band: the FP32 distance of cell-relative coordinates
    // (each below w/2 + skin/2 in magnitude) is within a few 1e-6 r_n^2 of
    // the exact one; candidates inside the band are decided in FP64
    double band = 1e-5 * a.rn2 + 1e-5;
    a.rn2_lo = (float)(a.rn2 - band);
    a.rn2_hi = (float)(a.rn2 + band);
    a.ushift = plan.ushift;
    a.ushiftf = (float)plan.ushift;
    a.thr2 = 0.25 * skin * skin;
    a.thr2f = (float)(a.thr2 * (1.0 - 1e-5));
    a.close2 = 0.08;
    a.close2f = 0.08f;
    // |f_d| = (f/r) |d_d| < (f/r) r_c for an interacting pair; 2000 leaves
    // room for the rounding of the product below 2^11
    a.fix_small_fr = (float)(2000.0 / std::sqrt(a.rc2));
    // shell bins: k skin / kShellBins above r_c.  The margin covers the FP32
    // rounding of the build distances, of the displacement bound and of the
    // step's distance test (each a few units of 1e-7 r_n).
    a.rcf = (float)rc;
    a.shell_inv = skin > 0.0 ? (float)(kShellBins / skin) : 0.0f;
    a.shell_eps = (float)(1e-4 * rn);
}

}  // namespace md
