// Batched operator applications over many right-hand sides and operators.
#pragma once

#include <vector>

#include "qxd_internal.cuh"

namespace qxd {

constexpr int BATCH_MAXR = 8;  // right-hand sides per site in one group

struct BatchItem {
    qxd_lattice* lat;
    const void* in;
    void* out;
};

// out_i = D_i in_i for all items (native layout, precision prec) in one
// launch; nr right-hand sides per site (0: autotuned and remembered)
int dw_batch(const std::vector<BatchItem>& items, int prec, int nr, cudaStream_t st);
// autotuned choice for a volume, 0 if not tuned yet
int dw_batch_tuned_nr(int prec, int volume);

}  // namespace qxd
