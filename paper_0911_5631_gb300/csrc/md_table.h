// md_table.h -- addresses of the kernels of one precision form, handed from
// the kernel translation units to the host runtime (graph nodes and stream
// launches take kernels by address).
#pragma once

namespace md {

template <class P>
struct KernelTable {
    void* set_state;
    void* bin;
    void* scan_apply;
    void* scatter;
    void* cellsort;
    void* gather;
    void* commit;
    void* build;     // thread per atom
    void* build_rows;  // the same, lists with each atom's entries contiguous (W transposed)
    void* build_direct;  // the same for lists longer than its stage: entries written as found
    void* build_wc;  // warp per home cell (warp-cooperative)
    void* rebuild_done;
    void* cond;
    void* kickdrift;
    void* step_tail;        // the step's closing work as a node of its own
    void* step_tail_final;
    void* step_list;
    void* step_list_final;
    void* step_cells;
    void* step_cells_final;
    void* finalize;
    void* get_state;
    void* get_forces;
    void* get_cells;
    void* reset_counters;
    void* clear_overflow;
    void* selftest;
    void* rescale;
    void* count_reads;
    void* spin;
    void* ensemble;  // mixed form only (nullptr for FP64)
    // step-kernel variants of the paper's ablations, mixed list form only
    // ({plain step, final step}; index = the MD_VARIANT_* bit position)
    void* step_var[4][2];
};

template <class P>
KernelTable<P> make_kernel_table();

}  // namespace md
