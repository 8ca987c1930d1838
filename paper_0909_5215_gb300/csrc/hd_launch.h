// hd_launch.h -- host-side launchers of the kernels in hd_kernels.cu.  Every
// launcher queues work on stream s and returns at once.
#pragma once
#include <cuda_runtime.h>

#include "hd_internal.cuh"

namespace hd {

void launch_init(const Dev &D, const int *draw_vel, cudaStream_t s);
void launch_rebuild(const Dev &D, cudaStream_t s);            // 5 kernels, flag-gated per replica
void launch_rebuild_prep(const Dev &D, cudaStream_t s);       // the first 4: plan, clear, bin, cell sort
void launch_nlist(const Dev &D, cudaStream_t s);              // the 5th: rows from the cells
// energy: also compute per-atom LJ energies (observables only; not needed by the dynamics)
void launch_pair(const Dev &D, bool quench, bool energy, cudaStream_t s);
void launch_scalar(const Dev &D, int mode, cudaStream_t s);
void launch_update(const Dev &D, int mode, cudaStream_t s);
void launch_obs(const Dev &D, cudaStream_t s);
void launch_nhc(const Dev &D, int mode, cudaStream_t s);          // the chain between two kicks, per replica
void launch_eig(const Dev &D, cudaStream_t s);                    // epsilon (Lanczos) and grad epsilon (hd_eig.cu)
void launch_qinit(const Dev &Q, const Dev &M, cudaStream_t s);
void launch_qiter(const Dev &Q, int max_iter, cudaStream_t s);  // 8 kernels
void launch_qdisp(const Dev &Q, cudaStream_t s);
void launch_adopt(const Dev &Q, const Dev &M, const int *adopt, cudaStream_t s);
size_t nl_smem_bytes(const Dev &D, int nwarps);                  // dynamic shared memory of the list build
// allow that much on the kernels that build lists; *nl_blocks_per_sm: resident row-build CTAs per SM
cudaError_t nl_configure(const Dev &D, int *nl_blocks_per_sm);
int persist_blocks_per_sm(const Dev &D);                          // resident CTAs of the persistent kernel
cudaError_t launch_persist(const Dev &D, int grid, int nsteps, cudaStream_t s);  // cooperative, n steps

}  // namespace hd
