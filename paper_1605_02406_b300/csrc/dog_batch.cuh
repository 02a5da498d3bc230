// dog_batch.cuh -- batched frame kernels: one launch per phase of the frame (Alg. 1-7) over
// the tiles of several independent filters.
//
// Each filter's parameters and buffer table (BatchFilter) lie in a slot of its own
// workspace.  A launch gets, by value, the slots of the filters that take part in the phase
// and the prefix of their block counts: block b belongs to filter k with
// first[k] <= b < first[k + 1] and acts as that filter's block b - first[k].  The block
// copies the filter's description into shared memory and runs the same per-block code as the
// single-filter kernel, so every filter's results equal those of its own dog_step.
#pragma once
#include "dog_kernels.cuh"

namespace dog {

constexpr int BATCH_MAX = 128;

struct BatchFilter {
  KParams P;
  DevBufs B;
  uint32_t count_ct;   // sort tiles per counting block
  uint32_t birth_grid; // newborn slot blocks
};
static_assert(sizeof(BatchFilter) <= 1024, "a filter's description fits its 1 KB slot");

struct BatchArgs {
  uint32_t n;                      // filters in this launch
  uint32_t first[BATCH_MAX + 1];   // first block of each, first[n] = blocks in all
  const BatchFilter *f[BATCH_MAX]; // their descriptions (device)
};

struct BatchBlock {
  uint32_t k, blk, nblk;
};

// the filter of this block (last k with first[k] <= blockIdx.x), its block and block count
__device__ __forceinline__ BatchBlock batch_block(const BatchArgs &A) {
  const uint32_t b = blockIdx.x;
  uint32_t lo = 0, hi = A.n - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (A.first[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return BatchBlock{lo, b - A.first[lo], A.first[lo + 1] - A.first[lo]};
}

// the block's filter description into shared memory (all threads; ends with a barrier)
__device__ __forceinline__ void batch_copy(BatchFilter &dst, const BatchFilter *src) {
  const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
  uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
  for (uint32_t i = threadIdx.x; i < sizeof(BatchFilter) / 4; i += blockDim.x) d[i] = __ldg(s + i);
  __syncthreads();
}

#define DOG_BATCH_PROLOGUE          \
  __shared__ BatchFilter s_bf;      \
  const BatchBlock bb = batch_block(A); \
  batch_copy(s_bf, A.f[bb.k]);      \
  const KParams &P = s_bf.P;        \
  const DevBufs &B = s_bf.B

__global__ void kb_ego_warp(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  ego_warp_body(P, B, bb.blk, bb.nblk);
}

__global__ void __launch_bounds__(PRED_BLOCK) kb_predict(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  predict_body(P, B, bb.blk);
}

// the key and value arrays that pass p of a filter's sort reads and writes
struct SortIO {
  const uint32_t *kin, *vin;
  uint32_t *kout, *vout;
};
__device__ __forceinline__ SortIO sort_io(const KParams &P, const DevBufs &B, int p) {
  SortIO io;
  io.kin = p == 0 ? B.key_pred : (p == 1 ? B.key_t0 : B.key_t1);
  io.vin = p == 0 ? nullptr : (p == 1 ? B.val_t0 : B.val_t1);
  const bool last = p == P.passes - 1;
  io.kout = last ? B.key_sorted : (p == 0 ? B.key_t0 : B.key_t1);
  io.vout = last ? B.perm : (p == 0 ? B.val_t0 : B.val_t1);
  return io;
}

__global__ void __launch_bounds__(COUNT_BLOCK) kb_sort_count(const __grid_constant__ BatchArgs A, int pass) {
  DOG_BATCH_PROLOGUE;
  sort_count_body(P, B, sort_io(P, B, pass).kin, pass, s_bf.count_ct, bb.blk);
}

template <int OFF_PER>
__global__ void __launch_bounds__(OFF_BLOCK, OFF_PER <= 4 ? 8 : 1) kb_sort_offsets(const __grid_constant__ BatchArgs A,
                                                                                   int pass) {
  DOG_BATCH_PROLOGUE;
  sort_offsets_body<OFF_PER>(P, B, pass, bb.blk);
}

__global__ void __launch_bounds__(SORT_BLOCK, 2) kb_sort_pass(const __grid_constant__ BatchArgs A, int pass) {
  DOG_BATCH_PROLOGUE;
  const SortIO io = sort_io(P, B, pass);
  sort_pass_body(P, B, io.kin, io.vin, io.kout, io.vout, pass, bb.blk);
}

template <bool RADAR>
__global__ void __launch_bounds__(SEG_BLOCK) kb_segsum(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  segsum_body<RADAR>(P, B, bb.blk);
}

__global__ void __launch_bounds__(SEG_BLOCK, 5) kb_segsum_lidar(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  segsum_lidar_body(P, B, bb.blk);
}

template <bool RADAR>
__global__ void __launch_bounds__(CELL_BLOCK) kb_cell(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  cell_body<RADAR>(P, B, bb.blk);
}

// the newborn-mass scan (SETUP = false) or the joint-weight CDF scan (true), one block each
template <bool SETUP>
__global__ void __launch_bounds__(SCAN_BLOCK) kb_scan_tiles(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  (void)bb;
  if (SETUP)
    scan_tiles_body<true>(B.cdf_tile, nullptr, P.tiles_norm, B.cdf_incl, nullptr, &B.ctl->W_total, nullptr, P,
                          B.ctl);
  else
    scan_tiles_body<false>(B.tile_q, B.tile_n, P.tiles_cell, B.tile_qin, B.tile_nin, &B.ctl->R_total,
                           &B.ctl->n_birth_cells, P, B.ctl);
}

template <bool RADAR>
__global__ void __launch_bounds__(BPREP_BLOCK) kb_birth_prep(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  birth_prep_body<RADAR>(P, B, bb.blk);
}

template <bool RADAR>
__global__ void __launch_bounds__(BIRTH_BLOCK) kb_birth(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  birth_body<RADAR>(P, B, bb.blk);
}

__global__ void __launch_bounds__(NORM_BLOCK) kb_normalise_radar(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  normalise_body<true>(P, B, bb.blk);
}

__global__ void __launch_bounds__(NORM_BLOCK, 4) kb_rmsum(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  rmsum_body(P, B, bb.blk);
}

__global__ void __launch_bounds__(NORM_BLOCK, 8) kb_normalise_lidar(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  normalise_lidar_body(P, B, bb.blk);
}

__global__ void __launch_bounds__(256) kb_moments(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  moments_body(P, B, bb.blk, bb.nblk);
}

__global__ void __launch_bounds__(RES_BLOCK, 5) kb_resample(const __grid_constant__ BatchArgs A) {
  DOG_BATCH_PROLOGUE;
  resample_body(P, B, bb.blk);
}

#undef DOG_BATCH_PROLOGUE

}  // namespace dog
