// Host-visible launchers of the support kernels (bd_support.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "bd_device.cuh"

namespace bdra {

cudaError_t run_exp1(const ChainDev* chains, const int32_t* spring_chain, int64_t M, uint32_t k0,
                     uint32_t k1, uint32_t chain_base, double* exp1, cudaStream_t st);
cudaError_t run_set_bonds(bool f64, const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                          const double* pos, void* state, cudaStream_t st);
cudaError_t run_spawn(bool f64, const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                      void* state, cudaStream_t st);
cudaError_t run_positions(bool f64, const ChainDev* chains, const int64_t* pair_off, int n_chains,
                          int64_t n_pairs, int all_slots, const void* state, double* out,
                          cudaStream_t st);
// The fold kernel (one thread per (window, spring); FoldParams by value) for
// graph kernel nodes.
const void* rsf_fold_func();
int rsf_fold_threads();
cudaError_t run_window_criteria(const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                                const double* rsf_hist, const double* tsf_hist, int64_t w0, int64_t w1, int S, double dt,
                                int thr_mask, int bell_mask, const double* exp1, double* lam,
                                int64_t* first_thr, int64_t* first_bell, cudaStream_t st);
int64_t event_blocks(int64_t M);
cudaError_t run_events(const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                       const int64_t* first_thr, const int64_t* first_bell, int64_t* block_scratch,
                       bd_event* out, int64_t capacity, cudaStream_t st);
cudaError_t run_log_survival(const ChainDev* chains, int n_chains, int64_t M, const double* lam,
                             double* out, cudaStream_t st);
cudaError_t run_adj_seed(const ChainDev* chains, const int32_t* spring_chain, int64_t M,
                         const double* rsf_hist, int64_t w_lo, int64_t n_w,
                         const double* grad_rsf, const double* grad_log_surv, int S, double dt,
                         double* G, cudaStream_t st);
cudaError_t run_normals(bool f64, int64_t n, const uint32_t* ctr, const StepParams& p, double* out,
                        cudaStream_t st);

}  // namespace bdra
