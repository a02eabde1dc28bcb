// akmc_launch.h -- host-side launchers of the libakmc kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include "akmc_device.cuh"

namespace akmc {

void launch_setup_model(ModelDev* M, int32_t* batch_status, int has_eam, int n_rho, cudaStream_t st);
// `list` (device, nullable): the voxel indices to work on; NULL means all.
void launch_place(VoxelDev* vox, int n_vox, const int32_t* list, cudaStream_t st);
cudaError_t launch_batch_load(VoxelDev* vox, const double* io, int n, int has_t, int has_n, cudaStream_t st);
cudaError_t launch_voxel_load(VoxelDev* V, const double* io, cudaStream_t st);
cudaError_t launch_batch_read(const VoxelDev* vox, double* io, int n, cudaStream_t st);
// io[v] = W, io[n+v] = M_hat, io[2n+v] = E_hat of voxel v (workload proxy, Eq. 10)
cudaError_t launch_proxy(const VoxelDev* vox, const ModelDev* M, double* io, int n, cudaStream_t st);

// Density tiles: cells [x0,x0+kTX) x [y0,y0+kTY) x [z0,z0+kTZ) of one voxel.
constexpr int kTX = 32, kTY = 16, kTZ = 16, kHalo = 2;
// Strips (voxels with L <= kStripMaxL): item (voxel, y0, z0, tz | vec << 16 | ty << 17)
// covers rows [y0, y0+ty) of planes [z0, z0+tz); vec = 16-byte aligned rows;
// ty = density_strip_rows(L); a strip of a voxel of edge L needs
// density_strip_smem(L) bytes of dynamic shared memory (strip_dyn: the batch maximum).
constexpr int kStripMaxL = 256;
int density_strip_rows(int L);
size_t density_strip_smem(int L);
cudaError_t launch_density(const VoxelDev* vox, const ModelDev* M, const Tables* tab, const int4* tiles,
                           int n_tiles, const int4* strips, int n_strips, size_t strip_dyn, cudaStream_t st);

size_t step_dyn_smem(int max_nv, int max_P, int win);
cudaError_t launch_rate_tables(VoxelDev* vox, int n_vox, const ModelDev* M, const int32_t* list,
                               cudaStream_t st);
cudaError_t launch_step(const BatchArgs& a, int warps, int grid, cudaStream_t st);
cudaError_t launch_rebuild(const BatchArgs& a, int warps, const int32_t* list, int n_list, cudaStream_t st);
int step_occupancy(int warps, int max_nv, int max_P, int win);
// Synchronous sublattice supersteps of one voxel: sl_prepare sets the kernel's
// shared-memory limit (once per call sequence, outside any capture);
// launch_sublattice runs superstep k over n_sectors = (L/sector_cells)^3 CTAs.
// stale[nv] (zeroed by the caller at the start of a call sequence) tracks which
// vacancies' stored rates are out of date.
cudaError_t sl_prepare(const BatchArgs& a);
cudaError_t launch_sublattice(const BatchArgs& a, int vid, uint32_t k, int sector_cells, int n_sectors,
                              double window, int32_t* stale, cudaStream_t st);
// Asynchronous form: n supersteps from k0 in one cooperative launch of
// min(n_sectors, resident CTAs) CTAs with per-sector readiness counters
// done[n_sectors] (zeroed by the caller) and an abort word; skip_sector >= 0
// (test hook) leaves one sector unprocessed; grid_out gets the grid size.
cudaError_t launch_sublattice_async(const BatchArgs& a, int vid, uint32_t k0, uint32_t n, int sector_cells,
                                    int n_sectors, double window, int32_t* done, int32_t* abort_flag,
                                    int32_t* stale, int skip_sector, int n_sm, int* grid_out, cudaStream_t st);

const Tables& host_tables();   // stencil tables built on the host
void set_last_error(const char* msg);   // text returned by akmc_last_error() on this thread
cudaError_t launch_cluster(const VoxelDev* vox, int voxel, int N, const Tables* tab, int mode,
                           int32_t* labels, int32_t* sizes, unsigned long long* hist, cudaStream_t st);

}  // namespace akmc
