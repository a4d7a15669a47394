// smc_host.h -- host-side state of a sampler handle, shared by the C-ABI
// translation units (smc_api.cu: single samplers; smc_batch.cu: batches).
#pragma once

#include <string>

#include "smc_internal.cuh"
#include "smc_kernels.h"

namespace smc {

// Byte offsets of the stateful sampler's workspace.
struct Layout {
  size_t st, tg, part, epart, qpart, cbase, xpart, rs, rs_alt, wbuf, tile_src, gbar, lg_x, lg_y, lg_img, covpart, total;
  int qblocks, ntiles, cov_blocks;
};

// Blocks of the covariance kernel (each writes D(D+1)/2 partial sums).
constexpr int kCovMaxBlocks = 304;

}  // namespace smc

struct smc_sampler {
  smc_config cfg;
  int64_t n;
  int d;
  int dtype;
  size_t esize;
  void* x[2];
  void* lp[2];
  double* logw;
  char* ws;
  smc::Layout L;
  cudaStream_t stream;
  smc::DevState* st;
  smc::TargetDev* tg;
  double* part;
  uint64_t* qpart;
  uint64_t* cbase;
  void* xpart;
  int32_t* rs;
  int32_t* rs_alt;  // second run-start array (samplers created with SMC_FLAG_DEFER_REDISTRIBUTE), else NULL
  uint64_t* wbuf;
  int32_t* tile_src;
  int grid_p;
  int threads_p;  // block size of the particle kernels
  // FP32 logistic samplers: likelihood on the tensor cores (its own grid)
  bool lg_tc;
  int grid_lg;
  // FP32 Gaussian samplers (have_gp): the factor for the move / reweight
  // kernel's parameters, valid once gp_ready (smc::fetch_gp)
  smc::GaussParamsF32 gp;
  bool have_gp;
  bool gp_ready;
  // SMC_FLAG_DEFER_REDISTRIBUTE honoured: resampled rows are gathered by the next move
  bool defer;
  // FP64 sampler of one quantise block and one copy tile: smc_step runs its
  // iterations in one cooperative launch (k_iterate_small)
  bool small_iter;
  // CUDA graph of one iteration (with and without the covariance stage)
  cudaGraphExec_t g_iter[2];
  std::string err;
};

namespace smc {

ParticleArgs particle_args(const smc_sampler* h);
QuantArgs quant_args(const smc_sampler* h, int force, int32_t* ncopies);
RedistArgs redist_args(const smc_sampler* h, int force);
// Completes a deferred redistribution on h's stream (no-op without the flag).
cudaError_t materialize(smc_sampler* h);
// Makes h->gp valid (FP32 Gaussian samplers; synchronises h's stream the
// first time; not during stream capture).
cudaError_t fetch_gp(smc_sampler* h);
int sm_count();

}  // namespace smc

