// mrlt_tree.cuh -- host-side launcher of the tree kernels (private).
#pragma once
#include "mrlt_tree_dev.cuh"

namespace mrlt {

constexpr int MASS_BLOCKS = 64;

struct Launcher {
    Grid g;
    cudaStream_t st = nullptr;
    int* bc = nullptr; // compaction scratch, 2 ints per block over all levels
    long long n = 0;   // kernel launches issued

    void project(int l, int mode);
    void project_up(int hi, int lo, int mode); // levels hi..lo, fewer launches
    void leaf_copy(int lo, int hi, int from, int to); // leaves of levels lo..hi
    void mark_refinements(int la, long long it = -1); // it >= 0: check that the tree fits (halt)
    void apply_tree(int la);
    void compact(int lo, int hi);                      // leaf / node / tile lists of levels lo..hi
    void reflux(int lo, int hi);                       // coarse levels lo..hi
    void scale(int l);
    void scale_init();                                 // running max |q_v| := 1e-14
    void set_dt(double dt);                            // *g.dtp := dt
    void set_leaves(const int* keys, const double* vals, long long count); // leaf q^n and end values
    void store_finest(const double* src); // finest-level q^n from double data [v][cell]
    void slots_full(long long ntot);      // every cell of every level a node (a new solver's tree)
    // compacting copy of the nodes from `from` into the arrays of g (a new capacity)
    void renumber(const Grid& from, const int* counts_host, long long used);
    void count_refined(int la, int* out);   // *out = refinement flags of levels la..L-1
    void finite(int l);
    void mass(int l, double* part);
    void pack(int l, long long base, int* keys, double* vals);
    void uniform(double* T, uint8_t* us);
};

} // namespace mrlt
