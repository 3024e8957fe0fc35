// Launch-shape autotuning of the D kernels: the process-wide table of chosen
// shapes, keyed by lattice shape and precision.
#pragma once

#include <string>
#include <tuple>

#include "qxd_internal.cuh"

namespace qxd {

// launch shape of the full-lattice D: hop order (1: software-pipelined, FP32
// only; 0: plain), threads per block, x2 rows per sweep chunk; ms: the time
// of one application measured when the shape was chosen (0 if not timed)
struct DwShape {
    int pipelined;
    int threads;
    int rows;
    float ms;
};

// precision, qhat != 0, N0, N1, N2, N3, C* mask
using DwKey = std::tuple<int, int, int, int, int, int, unsigned>;

DwKey dw_key(const qxd_lattice* lat, int prec);
DwShape dw_default_shape(const qxd_lattice* lat, int prec);
bool dw_shape_get(const DwKey& key, DwShape* out);
void dw_shape_put(const DwKey& key, const DwShape& sh, const char* how);
bool autotune_enabled();
// the rhs-per-site choices of the batched D, as text lines (batch.cu)
void dw_batch_report(std::string& out);

}  // namespace qxd
