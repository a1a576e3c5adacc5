// Internal interface of the projector translation unit.
#pragma once
#include "common.cuh"

namespace inrct {

// Geometry passed by value to kernels (mirrors inrct_geom plus the grid side).
struct GeomDev {
  int kind, N, V, A, B;
  double du, dv, sod, sdd, angle0, span;
};

int check_geom(const inrct_geom* geom, const inrct_grid* grid);
int64_t num_rays(const inrct_geom* geom);
size_t project_ws_bytes(const inrct_geom* geom, const inrct_grid* grid);
size_t backproject_ws_bytes(const inrct_geom* geom, const inrct_grid* grid);
int project_impl(const inrct_geom* geom, const inrct_grid* grid, const float* image, float* sino,
                 const float* y, float* resid, double* loss_out, void* ws, size_t ws_bytes,
                 cudaStream_t st);
int backproject_impl(const inrct_geom* geom, const inrct_grid* grid, const float* sino, float* image,
                     void* ws, size_t ws_bytes, cudaStream_t st);

}  // namespace inrct
