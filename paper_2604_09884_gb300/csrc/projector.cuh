// Internal interface of the projector translation unit.
#pragma once
#include "common.cuh"

namespace inrct {

// Geometry passed by value to kernels (mirrors inrct_geom plus the grid side).
struct GeomDev {
  int kind, N, V, A, B;
  double du, dv, sod, sdd, angle0, span;
};

// Cache seal of a geometry's ray tables in a workspace (see trig_kernel in projector.cu).
struct TabSeal {
  unsigned long long fp;  // fingerprint of the geometry and placement of the completed tables
  unsigned int skip;      // set by the first build kernel: the tables are valid, skip the build
  unsigned int done;      // blocks of the ray build that finished (the last one seals)
};

// Ray tables of one geometry (see projector.cu).
struct ProjTables {
  TabSeal* seal0;
  TabSeal* seal1;
  int4* tab0;
  int4* tab1;
  float* tab2;
  float2* views;
  double2* vtrig;
  double2* btrig;
};

// Launch shape of P and P^T for one geometry (see "Launch plans" in projector.cu).
struct ProjPlan {
  int seg;        // forward: ray segments per block
  int bp_splits;  // 2-D adjoint: view splits
  int zc;         // cone adjoint: voxels per thread along z
};
// The plan in use for a geometry; true when it came from the tuner.
bool plan_lookup(const inrct_geom* geom, const inrct_grid* grid, ProjPlan* out);
void plan_reset();
// Pins a plan for a geometry after checking it is one of the candidates.
int plan_set(const inrct_geom* geom, const inrct_grid* grid, const ProjPlan& p);
size_t tune_ws_bytes(const inrct_geom* geom, const inrct_grid* grid);
// Times every candidate plan on st (synchronises it) and keeps the fastest.
int tune_impl(const inrct_geom* geom, const inrct_grid* grid, void* ws, size_t ws_bytes, cudaStream_t st,
              ProjPlan* out);

int check_geom(const inrct_geom* geom, const inrct_grid* grid);
size_t tables_bytes(const inrct_geom* geom);
int build_tables(const inrct_geom* geom, const inrct_grid* grid, void* ws, size_t ws_bytes,
                 ProjTables* t, cudaStream_t st);
int64_t num_rays(const inrct_geom* geom);
// Workspace of one call; with_tables = false when the caller passes prebuilt tables.
size_t project_ws_bytes(const inrct_geom* geom, const inrct_grid* grid, bool with_tables = true);
size_t backproject_ws_bytes(const inrct_geom* geom, const inrct_grid* grid, bool with_tables = true);
int project_impl(const inrct_geom* geom, const inrct_grid* grid, const float* image, float* sino,
                 const float* y, float* resid, double* loss_out, void* ws, size_t ws_bytes,
                 cudaStream_t st, const ProjTables* pre = nullptr);
int backproject_impl(const inrct_geom* geom, const inrct_grid* grid, const float* sino, float* image,
                     void* ws, size_t ws_bytes, cudaStream_t st, const ProjTables* pre = nullptr);
int project_noalloc_impl(const inrct_geom* geom, const inrct_grid* grid, const float* image,
                         float* sino, const float* y, float* resid, double* loss_out, cudaStream_t st);

}  // namespace inrct
