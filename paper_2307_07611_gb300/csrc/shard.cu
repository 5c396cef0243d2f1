// shard.cu -- host-side partition of independent blocks or matrices over the ranks of a
// multi-GPU job (one process per GPU).  The blocks of a batched inverse (a block-Jacobi
// preconditioner's diagonal blocks) or the matrices of a batch are independent, so the
// job shards with no collective on the data path: every rank inverts the blocks it owns
// and the results stay on its GPU.
//
// Cost of a block of order m: m^3 (the recursive split of Section 4.1 does m^3/3 flops
// per inverse).  Blocks are assigned longest first to the rank with the smallest load so
// far (greedy LPT; ties go to the lower block index and the lower rank), which bounds
// the largest load by 4/3 of the optimum and, for thousands of blocks, brings every load
// within a fraction of a percent of the mean.  Deterministic: every rank computes the
// same assignment from the same sizes, so no exchange is needed.
#include <algorithm>
#include <numeric>
#include <queue>
#include <vector>

#include "internal.cuh"

extern "C" tri_status tri_batched_partition(int64_t count, const int64_t *sizes, int world, int32_t *owner,
                                            double *loads) {
    if (count < 0 || world < 1 || (count > 0 && (!sizes || !owner))) return TRI_ERR_ARG;
    for (int64_t i = 0; i < count; ++i)
        if (sizes[i] < 0) return TRI_ERR_ARG;
    std::vector<int64_t> order((size_t)count);
    std::iota(order.begin(), order.end(), (int64_t)0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return sizes[a] > sizes[b]; });
    using Load = std::pair<double, int>;   // (load, rank): smallest load, then smallest rank
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int r = 0; r < world; ++r) heap.push({0.0, r});
    std::vector<double> load((size_t)world, 0.0);
    for (int64_t i : order) {
        Load top = heap.top();
        heap.pop();
        const double m = (double)sizes[i];
        owner[i] = top.second;
        top.first += m * m * m;
        load[(size_t)top.second] = top.first;
        heap.push(top);
    }
    if (loads)
        for (int r = 0; r < world; ++r) loads[r] = load[(size_t)r];
    return TRI_OK;
}
