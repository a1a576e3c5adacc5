// Internal interface of the ramp filter (FLS loss, Sec. 2).
#pragma once
#include "common.cuh"

namespace inrct {
size_t ramp_ws_bytes(const inrct_geom* geom);
int ramp_filter_impl(const inrct_geom* geom, const inrct_grid* grid, const float* r, float* out,
                     double* loss_out, void* ws, size_t ws_bytes, cudaStream_t st);
}  // namespace inrct
