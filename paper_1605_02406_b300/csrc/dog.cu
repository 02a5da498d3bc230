// dog.cu -- host side of the C ABI declared in include/dog.h: parameter validation,
// workspace carving, the per-frame launch sequence (optionally captured once into a CUDA
// graph and replayed), checkpoint, intermediates and kernel profiling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/dog.h"
#include "dog_kernels.cuh"
#include "dog_batch.cuh"
#include "dog_eval.cuh"

using namespace dog;

namespace {

constexpr int MAX_KERNELS = 18;
constexpr size_t DOG_BATCH_GROUP_BYTES_DEFAULT = 0;  // one filter per branch
constexpr int PROFILE_RING = 1024;

struct Derived {
  uint32_t C;
  int key_bits, passes, dbits;
  uint32_t radix;
  uint32_t tiles_sort, tiles_seg, tiles_cell, tiles_norm;
};

int check_params(const dog_params *p, Derived *d) {
  if (!p) return DOG_ERR_INVALID_ARG;
  if (p->width <= 0 || p->height <= 0 || !(p->cell_size > 0.0f) || !std::isfinite(p->cell_size))
    return DOG_ERR_INVALID_ARG;
  if (p->num_particles == 0) return DOG_ERR_INVALID_ARG;
  const float probs[] = {p->p_S, p->p_B, p->alpha_free};
  for (float v : probs)
    if (!(v >= 0.0f && v <= 1.0f)) return DOG_ERR_INVALID_ARG;
  const float sds[] = {p->sigma_pos, p->sigma_vel, p->sigma_birth_vel};
  for (float v : sds)
    if (!(v >= 0.0f) || !std::isfinite(v)) return DOG_ERR_INVALID_ARG;
  if (!std::isfinite(p->sensor_x) || !std::isfinite(p->sensor_y)) return DOG_ERR_INVALID_ARG;
  const unsigned long long C = (unsigned long long)p->width * (unsigned long long)p->height;
  // C < 2^24 keeps the joint weight total (<= C cell masses of at most 1, scale 2^40) < 2^64
  if (C >= (1ull << 24)) return DOG_ERR_UNSUPPORTED;
  if (p->num_particles >= (1u << 25) || p->num_birth >= (1u << 25)) return DOG_ERR_UNSUPPORTED;
  d->C = (uint32_t)C;
  int bits = 1;
  while ((1ull << bits) < C) ++bits;
  d->key_bits = bits;
  d->passes = (bits + 10) / 11;
  d->dbits = (bits + d->passes - 1) / d->passes;
  d->radix = 1u << d->dbits;
  const uint32_t nu = p->num_particles, ntot = nu + p->num_birth;
  d->tiles_sort = (nu + SORT_TILE - 1) / SORT_TILE;
  d->tiles_seg = (nu + SEG_TILE - 1) / SEG_TILE;
  d->tiles_cell = (d->C + CELL_TILE - 1) / CELL_TILE;
  d->tiles_norm = (ntot + NORM_TILE - 1) / NORM_TILE;
  return DOG_OK;
}

// Carve every array out of the workspace (base == nullptr: only count).  Returns bytes.
size_t carve(const dog_params &p, const Derived &d, char *base, DevBufs *B) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> void * {
    off = (off + 255) & ~(size_t)255;
    void *ptr = base ? base + off : nullptr;
    off += bytes;
    return ptr;
  };
  const size_t nu = p.num_particles, nb = p.num_birth, C = d.C;
  const bool record = (p.flags & DOG_RECORD) != 0;
  B->ctl = (DevCtl *)take(sizeof(DevCtl));
  float4 **ps[] = {&B->As, &B->Os};
  for (auto q : ps) *q = (float4 *)take(16 * nu);
  B->Bsrc = (uint32_t *)take(4 * nu);
  B->stage = (float4 *)take(16 * (nu > nb ? nu : nb));
  float **pf[] = {&B->Bw, &B->Aw, &B->Ow, &B->wn};
  for (auto q : pf) *q = (float *)take(4 * nu);
  uint32_t **pu[] = {&B->key_pred, &B->key_sorted, &B->perm};
  for (auto q : pu) *q = (uint32_t *)take(4 * nu);
  B->key_t0 = B->val_t0 = B->key_t1 = B->val_t1 = nullptr;
  // DOG_AUTOTUNE: also the ping-pong buffers of a sort with one pass more
  const int max_passes = (p.flags & DOG_AUTOTUNE) ? (d.passes < 3 ? d.passes + 1 : 3) : d.passes;
  if (max_passes >= 2) {
    B->key_t0 = (uint32_t *)take(4 * nu);
    B->val_t0 = (uint32_t *)take(4 * nu);
  }
  if (max_passes >= 3) {
    B->key_t1 = (uint32_t *)take(4 * nu);
    B->val_t1 = (uint32_t *)take(4 * nu);
  }
  B->bs = (float4 *)take(16 * (nb ? nb : 1));
  B->bw = (float *)take(4 * (nb ? nb : 1));
  B->bcell = record ? (uint32_t *)take(4 * (nb ? nb : 1)) : nullptr;
  B->bassoc = record ? (uint32_t *)take(4 * (nb ? nb : 1)) : nullptr;
  float **pc[] = {&B->mF, &B->zO, &B->zF, &B->pA, &B->zv, &B->sgv, &B->mO, &B->rho_p, &B->rho_b,
                  &B->pO, &B->mean_x, &B->mean_y, &B->var_x, &B->var_y, &B->cov, &B->mpred,
                  &B->muA, &B->muU, &B->paeff};
  for (auto q : pc) *q = (float *)take(4 * C);
  B->mF_warp = (p.flags & DOG_EGO) ? (float *)take(4 * C) : nullptr;
  B->mF_in = (p.flags & DOG_EGO) ? B->mF_warp : B->mF;
  B->rb_pred = (p.flags & DOG_FULL) ? (float *)take(4 * C) : nullptr;
  B->csum = (CellSum *)take(sizeof(CellSum) * C);
  B->cmom = (CellMom *)take(sizeof(CellMom) * C);
  B->g_stage = (float *)take(4 * 5 * C);
  B->c_stage = (float *)take(4 * (10 * C + 64));
  B->A = (unsigned long long *)take(8 * C);
  B->cstart = (uint32_t *)take(4 * C);
  B->cend = (uint32_t *)take(4 * C);
  const size_t CL = (size_t)d.tiles_cell * CELL_TILE;  // per-tile lists of birth cells
  B->bl_cell = (uint32_t *)take(4 * CL);
  B->bl_R = (unsigned long long *)take(8 * CL);
  B->bl_first = (uint32_t *)take(4 * (CL + 1));
  B->bl_gcell = (uint32_t *)take(4 * CL);
  B->bl_nA = (uint32_t *)take(4 * CL);
  B->bl_wA = (float *)take(4 * CL);
  B->bl_wUA = (float *)take(4 * CL);
  B->birth_block_entry = (uint32_t *)take(4 * ((nb + BIRTH_SLOTS - 1) / BIRTH_SLOTS + 1));
  B->hist = (uint32_t *)take(4 * 2048 * (size_t)max_passes);
  B->dcnt = (uint32_t *)take(4 * (size_t)d.passes * d.tiles_sort * d.radix);
  B->S_piece = (unsigned long long *)take(8 * C);
  B->A_piece = (unsigned long long *)take(8 * C);
  B->Mx = (unsigned long long *)take(8 * 5 * C);
  B->Pf = (float *)take(4 * 20 * (size_t)d.tiles_seg);
  B->tile_whole = (uint32_t *)take(4 * (size_t)d.tiles_seg);
  B->cross_t1 = (uint32_t *)take(4 * C);
  B->tile_q = (unsigned long long *)take(8 * (size_t)d.tiles_cell);
  B->tile_qin = (unsigned long long *)take(8 * (size_t)d.tiles_cell);
  B->tile_n = (uint32_t *)take(4 * (size_t)d.tiles_cell);
  B->tile_nin = (uint32_t *)take(4 * (size_t)d.tiles_cell);
  B->cdf_tile = (unsigned long long *)take(8 * (size_t)d.tiles_norm);
  B->cdf_incl = (unsigned long long *)take(8 * (size_t)d.tiles_norm);
  B->batch_slot = (unsigned char *)take(1024);
  return (off + 255) & ~(size_t)255;
}

const char *KNAMES[MAX_KERNELS] = {"k_ego_warp", "k_predict", "k_sort_offsets0", "k_sort_pass0",
                                   "k_sort_count1", "k_sort_offsets1", "k_sort_pass1",
                                   "k_sort_count2", "k_sort_offsets2", "k_sort_pass2",
                                   "k_segsum", "k_cell", "k_scan_births", "k_birth_prep", "k_birth",
                                   "k_normalise", "k_scan_cdf", "k_resample"};

}  // namespace

struct dog_filter {
  dog_params p;
  Derived d;
  KParams K;
  DevBufs B;
  cudaStream_t st;
  char *ws;
  size_t ws_bytes;
  bool has_grid = false, radar = false;
  bool dt_valid = false;
  float dt = 0.0f;
  uint32_t frame = 0;  // host mirror of DevCtl::frame
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  bool use_graph = true;
  // profiling
  bool profile = false;
  std::vector<cudaEvent_t> ev;  // PROFILE_RING * (MAX_KERNELS + 1)
  int ring_head = 0, ring_count = 0;
  int nk = 0;
  int birth_grid = 1;
  uint32_t count_ct = 1;  // sort tiles per k_sort_count block
  // ego motion for the next step (DOG_EGO): on, cos, sin, dx, dy
  bool ego_on = false;
  float ego_c = 1.0f, ego_s = 0.0f, ego_dx = 0.0f, ego_dy = 0.0f;
  // host I/O overlapped with compute: grid uploads and cell read-backs on their own streams
  cudaStream_t h2d = nullptr, d2h = nullptr;
  // the second branch of a frame (normalisation beside the newborn chain)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_mjoin = nullptr;
  cudaEvent_t ev_h2d = nullptr, ev_stage_free = nullptr, ev_snap = nullptr, ev_d2h = nullptr;
  bool d2h_pending = false;
  uint32_t *d2h_err = nullptr;  // pinned host word: error bits of the frame being read back
  // batched launches: the batch whose view of this filter its workspace slot holds, and a
  // counter of changes of the launch configuration (sort passes, digit width, count tiles)
  const void *slot_owner = nullptr;
  uint32_t cfg_version = 0;
};

namespace {

thread_local const char *t_last_cuda_error = "";

int cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return DOG_OK;
  t_last_cuda_error = cudaGetErrorString(e);
  (void)cudaGetLastError();
  return DOG_ERR_CUDA;
}

// k_sort_offsets of pass p with the register run that covers the sort tiles
void launch_offsets(const KParams &K, const DevBufs &B, int p, cudaStream_t st) {
  switch (offsets_per(K.tiles_sort)) {
    case 4: k_sort_offsets<4><<<K.radix, OFF_BLOCK, 0, st>>>(K, B, p); break;
    case 8: k_sort_offsets<8><<<K.radix, OFF_BLOCK, 0, st>>>(K, B, p); break;
    default: k_sort_offsets<16><<<K.radix, OFF_BLOCK, 0, st>>>(K, B, p); break;
  }
}

#define DOG_CUDA(x)                              \
  do {                                           \
    const cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

// the normalisation of the persistent sources (Alg. 4), on stream st
int enqueue_normalise(dog_filter *f, bool radar, cudaStream_t st) {
  const KParams &K = f->K;
  const DevBufs &B = f->B;
  const uint32_t tiles = (K.nu + NORM_TILE - 1) / NORM_TILE;
  if (radar) k_normalise<true><<<tiles, NORM_BLOCK, 0, st>>>(K, B);
  else k_normalise_lidar<<<tiles, NORM_BLOCK, 0, st>>>(K, B);
  return cuda_fail(cudaGetLastError());
}

// the radar filter's velocity moments (Alg. 6) from the normalised weights, on stream st
int enqueue_radar_moments(dog_filter *f, cudaStream_t st) {
  const KParams &K = f->K;
  const DevBufs &B = f->B;
  const uint32_t tiles = (K.nu + NORM_TILE - 1) / NORM_TILE;
  k_rmsum<<<tiles, NORM_BLOCK, 0, st>>>(K, B);
  k_moments<<<(K.C + 255) / 256 < 2368u ? (K.C + 255) / 256 : 2368u, 256, 0, st>>>(K, B);
  return cuda_fail(cudaGetLastError());
}

// the kernels of one frame, in order; ev (optional, profiling) are recorded around each
// kernel, which are then issued one after the other on the filter's stream; otherwise the
// normalisation runs on a second branch beside the newborn chain, and the radar filter's
// velocity moments continue that branch beside the CDF scan and the resampling, joined at
// the end of the frame
int enqueue_frame(dog_filter *f, bool radar, cudaEvent_t *ev) {
  const KParams &K = f->K;
  const DevBufs &B = f->B;
  cudaStream_t st = f->st;
  int k = 0;
  auto mark = [&]() {
    if (ev) cudaEventRecord(ev[k], st);
  };
  mark();
  // no frame tick: the sort passes and the CDF scan reset what the frame accumulates into
  if (K.flags & DOG_EGO) {
    k_ego_warp<<<592, 256, 0, st>>>(K, B);
    ++k; mark();
  }
  const uint32_t pred_grid = (K.nu + PRED_TILE - 1) / PRED_TILE;
  k_predict<<<pred_grid, PRED_BLOCK, 4u * K.passes * K.radix, st>>>(K, B);
  ++k; mark();
  const size_t ssm = sort_smem_bytes(K.radix);
  const uint32_t *kin = B.key_pred, *vin = nullptr;
  for (int p = 0; p < K.passes; ++p) {
    uint32_t *kout, *vout;
    if (p == K.passes - 1) {
      kout = B.key_sorted;
      vout = B.perm;
    } else if (p == 0) {
      kout = B.key_t0;
      vout = B.val_t0;
    } else {
      kout = B.key_t1;
      vout = B.val_t1;
    }
    if (p > 0) {
      k_sort_count<<<(K.tiles_sort + f->count_ct - 1) / f->count_ct, COUNT_BLOCK,
                     count_smem_bytes(K.radix, f->count_ct), st>>>(K, B, kin, p, f->count_ct);
      ++k; mark();
    }
    launch_offsets(K, B, p, st);
    ++k; mark();
    k_sort_pass<<<K.tiles_sort, SORT_BLOCK, ssm, st>>>(K, B, kin, vin, kout, vout, p);
    kin = kout;
    vin = vout;
    ++k; mark();
  }
  if (radar) k_segsum<true><<<K.tiles_seg, SEG_BLOCK, 0, st>>>(K, B);
  else k_segsum_lidar<<<K.tiles_seg, SEG_BLOCK, 0, st>>>(K, B);
  ++k; mark();
  if (radar) k_cell<true><<<K.tiles_cell, CELL_BLOCK, 0, st>>>(K, B);
  else k_cell<false><<<K.tiles_cell, CELL_BLOCK, 0, st>>>(K, B);
  ++k; mark();
  // the persistent sources' normalisation (and the radar moments) do not depend on the
  // newborn chain: outside profiling they run on a second branch from here on
  if (!ev) {
    DOG_CUDA(cudaEventRecord(f->ev_fork, st));
    DOG_CUDA(cudaStreamWaitEvent(f->aux, f->ev_fork, 0));
    int rc = enqueue_normalise(f, radar, f->aux);
    if (rc) return rc;
    DOG_CUDA(cudaEventRecord(f->ev_join, f->aux));
    if (radar) {
      rc = enqueue_radar_moments(f, f->aux);
      if (rc) return rc;
      DOG_CUDA(cudaEventRecord(f->ev_mjoin, f->aux));
    }
  }
  k_scan_tiles<false><<<1, SCAN_BLOCK, 0, st>>>(B.tile_q, B.tile_n, K.tiles_cell, B.tile_qin, B.tile_nin,
                                                 &B.ctl->R_total, &B.ctl->n_birth_cells, K, B.ctl);
  ++k; mark();
  if (radar) k_birth_prep<true><<<K.tiles_cell, BPREP_BLOCK, 0, st>>>(K, B);
  else k_birth_prep<false><<<K.tiles_cell, BPREP_BLOCK, 0, st>>>(K, B);
  ++k; mark();
  if (radar) k_birth<true><<<f->birth_grid, BIRTH_BLOCK, 0, st>>>(K, B);
  else k_birth<false><<<f->birth_grid, BIRTH_BLOCK, 0, st>>>(K, B);
  ++k; mark();
  if (!ev) {  // the normalisation ran on the second branch; the CDF scan waits for both
    DOG_CUDA(cudaStreamWaitEvent(st, f->ev_join, 0));
  } else {
    int rc = enqueue_normalise(f, radar, st);
    if (rc == DOG_OK && radar) rc = enqueue_radar_moments(f, st);  // timed with the normalisation
    if (rc) return rc;
  }
  ++k; mark();
  k_scan_tiles<true><<<1, SCAN_BLOCK, 0, st>>>(B.cdf_tile, nullptr, K.tiles_norm, B.cdf_incl, nullptr,
                                                &B.ctl->W_total, nullptr, K, B.ctl);
  ++k; mark();
  k_resample<<<K.tiles_norm, RES_BLOCK, 0, st>>>(K, B);
  ++k; mark();
  if (!ev && radar) DOG_CUDA(cudaStreamWaitEvent(st, f->ev_mjoin, 0));  // the moments' branch
  return cuda_fail(cudaGetLastError());
}

int read_err(dog_filter *f) {
  DevCtl h;
  DOG_CUDA(cudaMemcpyAsync(&h, f->B.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, f->st));
  DOG_CUDA(cudaStreamSynchronize(f->st));
  if (h.err) {
    const uint32_t zero = 0;
    DOG_CUDA(cudaMemcpyAsync(&f->B.ctl->err, &zero, 4, cudaMemcpyHostToDevice, f->st));
    DOG_CUDA(cudaStreamSynchronize(f->st));
    if (h.err & ERR_INPUT) return DOG_ERR_INPUT;
    return DOG_ERR_DEVICE;
  }
  return DOG_OK;
}

// zero the cell tags and the piece accumulators (needed whenever the frame counter is set
// to a value earlier frames may have used, and to drop whatever a failed frame left behind)
int reset_epochs(dog_filter *f) {
  const Derived &d = f->d;
  DevBufs &B = f->B;
  DOG_CUDA(cudaMemsetAsync(B.csum, 0, sizeof(CellSum) * (size_t)d.C, f->st));
  DOG_CUDA(cudaMemsetAsync(B.S_piece, 0, 8 * (size_t)d.C, f->st));
  DOG_CUDA(cudaMemsetAsync(B.A_piece, 0, 8 * (size_t)d.C, f->st));
  DOG_CUDA(cudaMemsetAsync(B.Mx, 0, 8 * 5 * (size_t)d.C, f->st));
  return DOG_OK;
}

// Records (x, y, vx, vy) <-> four plain float arrays, through the staging buffer
// (16 bytes per particle or newborn slot).
int unpack_records(dog_filter *f, const float4 *rec, size_t n, float *const dst[4], cudaMemcpyKind kd) {
  if (n == 0) return DOG_OK;
  float *scr = reinterpret_cast<float *>(f->B.stage);
  k_unpack<<<1024, 256, 0, f->st>>>(rec, (uint32_t)n, scr);
  DOG_CUDA(cudaGetLastError());
  for (int k = 0; k < 4; ++k)
    if (dst[k]) DOG_CUDA(cudaMemcpyAsync(dst[k], scr + k * n, 4 * n, kd, f->st));
  return DOG_OK;
}
int pack_records(dog_filter *f, float4 *rec, size_t n, const float *const src[4], cudaMemcpyKind kd) {
  float *scr = reinterpret_cast<float *>(f->B.stage);
  for (int k = 0; k < 4; ++k) DOG_CUDA(cudaMemcpyAsync(scr + k * n, src[k], 4 * n, kd, f->st));
  k_pack<<<1024, 256, 0, f->st>>>(scr, (uint32_t)n, rec);
  DOG_CUDA(cudaGetLastError());
  return DOG_OK;
}

cudaMemcpyKind kind_to(int mem) { return mem == DOG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }
cudaMemcpyKind kind_from(int mem) { return mem == DOG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }

}  // namespace

extern "C" {

const char *dog_last_cuda_error(void) { return t_last_cuda_error; }

int dog_eval_clusters(dog_filter *f, const int32_t *d_cell_object, uint32_t n_objects, long long *d_scratch,
                      double *d_stats) {
  if (!f || !d_cell_object || !d_scratch || !d_stats || n_objects == 0) return DOG_ERR_INVALID_ARG;
  DOG_CUDA(cudaMemsetAsync(d_scratch, 0, sizeof(long long) * 5 * (size_t)n_objects, f->st));
  const uint32_t grid = (f->d.C + EVAL_BLOCK - 1) / EVAL_BLOCK < 2048u ? (f->d.C + EVAL_BLOCK - 1) / EVAL_BLOCK : 2048u;
  k_eval_cluster_sums<<<grid, EVAL_BLOCK, 0, f->st>>>(f->K, f->B, d_cell_object, n_objects, d_scratch);
  k_eval_cluster_stats<<<(n_objects + 255) / 256, 256, 0, f->st>>>(d_scratch, n_objects, d_stats);
  return cuda_fail(cudaGetLastError());
}

int dog_eval_mahalanobis(dog_filter *f, const uint8_t *d_label, float min_occ, const float *d_thresholds,
                         uint32_t n_thresholds, unsigned long long *d_counts, float *d_m) {
  if (!f || !d_label || !d_counts || (n_thresholds > 0 && !d_thresholds)) return DOG_ERR_INVALID_ARG;
  if (n_thresholds > 4096) return DOG_ERR_UNSUPPORTED;
  const size_t nb = 2 * ((size_t)n_thresholds + 1);
  DOG_CUDA(cudaMemsetAsync(d_counts, 0, sizeof(unsigned long long) * nb, f->st));
  const uint32_t grid = (f->d.C + EVAL_BLOCK - 1) / EVAL_BLOCK < 1184u ? (f->d.C + EVAL_BLOCK - 1) / EVAL_BLOCK : 1184u;
  k_eval_mahalanobis<<<grid, EVAL_BLOCK, 4 * nb, f->st>>>(f->K, f->B, d_label, min_occ, d_thresholds,
                                                           n_thresholds, d_counts, d_m);
  return cuda_fail(cudaGetLastError());
}

const char *dog_error_string(int code) {
  switch (code) {
    case DOG_OK: return "ok";
    case DOG_ERR_INVALID_ARG: return "invalid argument";
    case DOG_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case DOG_ERR_CUDA: return "CUDA runtime error";
    case DOG_ERR_DEVICE: return "device-side consistency check failed";
    case DOG_ERR_INPUT: return "input outside its domain";
    case DOG_ERR_BAD_STATE: return "call not valid in the current state";
    case DOG_ERR_UNSUPPORTED: return "size beyond the supported maximum";
    default: return "unknown error";
  }
}

int dog_workspace_bytes(const dog_params *params, size_t *out_bytes) {
  if (!out_bytes) return DOG_ERR_INVALID_ARG;
  Derived d;
  const int rc = check_params(params, &d);
  if (rc) return rc;
  DevBufs B;
  *out_bytes = carve(*params, d, nullptr, &B);
  return DOG_OK;
}

int dog_kernels_per_step(const dog_filter *f) {
  if (!f) return 0;
  // + the radar filter's two moment kernels, + the ego-motion setting and warp
  return f->nk + (f->radar ? 2 : 0) + ((f->p.flags & DOG_EGO) ? 2 : 0);
}

static_assert(FLAG_EGO == DOG_EGO, "the kernels' ego flag is the ABI's");

int dog_set_ego_motion(dog_filter *f, float dx, float dy, float dyaw) {
  if (!f) return DOG_ERR_INVALID_ARG;
  if (!(f->p.flags & DOG_EGO)) return DOG_ERR_BAD_STATE;
  if (!std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dyaw)) return DOG_ERR_INVALID_ARG;
  f->ego_on = dx != 0.0f || dy != 0.0f || dyaw != 0.0f;
  f->ego_c = (float)std::cos((double)dyaw);
  f->ego_s = (float)std::sin((double)dyaw);
  f->ego_dx = dx;
  f->ego_dy = dy;
  return DOG_OK;
}

namespace {
// the pending ego motion into the control block, in stream order before the frame; it then
// returns to "none" for the frames after
int issue_ego(dog_filter *f, cudaStream_t st) {
  if (!(f->p.flags & DOG_EGO)) return DOG_OK;
  k_set_ego<<<1, 1, 0, st>>>(f->B.ctl, f->ego_on ? 1u : 0u, f->ego_c, f->ego_s, f->ego_dx, f->ego_dy);
  f->ego_on = false;
  f->ego_c = 1.0f;
  f->ego_s = f->ego_dx = f->ego_dy = 0.0f;
  return cuda_fail(cudaGetLastError());
}
}  // namespace

static void apply_cached_sort_cfg(dog_filter *f);

int dog_create(const dog_params *params, void *d_workspace, size_t workspace_bytes, void *cuda_stream,
               dog_filter **out) {
  if (!out || !d_workspace) return DOG_ERR_INVALID_ARG;
  *out = nullptr;
  Derived d;
  int rc = check_params(params, &d);
  if (rc) return rc;
  if (((uintptr_t)d_workspace & 255) != 0) return DOG_ERR_INVALID_ARG;
  DevBufs B;
  const size_t need = carve(*params, d, nullptr, &B);
  if (workspace_bytes < need) return DOG_ERR_WORKSPACE_TOO_SMALL;
  dog_filter *f = new (std::nothrow) dog_filter();
  if (!f) return DOG_ERR_INVALID_ARG;
  f->p = *params;
  f->d = d;
  f->st = (cudaStream_t)cuda_stream;
  f->ws = (char *)d_workspace;
  f->ws_bytes = workspace_bytes;
  carve(*params, d, f->ws, &f->B);
  KParams &K = f->K;
  K.W = params->width;
  K.H = params->height;
  K.C = d.C;
  K.s = params->cell_size;
  K.nu = params->num_particles;
  K.nu_b = params->num_birth;
  K.p_S = params->p_S;
  K.p_B = params->p_B;
  K.alpha = params->alpha_free;
  K.sigma_pos = params->sigma_pos;
  K.sigma_vel = params->sigma_vel;
  K.sigma_B = params->sigma_birth_vel;
  K.sensor_x = params->sensor_x;
  K.sensor_y = params->sensor_y;
  K.seed_lo = (uint32_t)params->seed;
  K.seed_hi = (uint32_t)(params->seed >> 32);
  K.flags = params->flags;
  K.passes = d.passes;
  K.dbits = d.dbits;
  K.radix = d.radix;
  K.tiles_sort = d.tiles_sort;
  K.tiles_seg = d.tiles_seg;
  K.tiles_cell = d.tiles_cell;
  K.tiles_norm = d.tiles_norm;
  f->nk = 8 + 3 * d.passes;
  f->profile = (params->flags & DOG_PROFILE) != 0;
  f->use_graph = !(params->flags & DOG_NO_GRAPH) && f->st != nullptr && !f->profile;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  f->birth_grid = (int)((params->num_birth + BIRTH_SLOTS - 1) / BIRTH_SLOTS);
  f->count_ct = count_tiles_per_block(d.tiles_sort, sms);
  if (f->birth_grid < 1) f->birth_grid = 1;
  apply_cached_sort_cfg(f);
  // the attribute is per kernel, shared by all filters: allow the largest digit's need
  cudaError_t e = cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sort_smem_bytes(2048));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sort_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)count_smem_bytes(2048, COUNT_TILES));
  if (e == cudaSuccess) e = cudaMemsetAsync(f->ws, 0, need, f->st);
  if (e == cudaSuccess) {
    k_init<<<sms * 8, 256, 0, f->st>>>(K, f->B);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f->h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f->d2h, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f->aux, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost(&f->d2h_err, 64);  // pinned: the copy stays asynchronous
  cudaEvent_t *evs[] = {&f->ev_h2d, &f->ev_stage_free, &f->ev_snap, &f->ev_d2h, &f->ev_fork, &f->ev_join, &f->ev_mjoin};
  for (auto q : evs)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(q, cudaEventDisableTiming);
  if (e == cudaSuccess && f->profile) {
    f->ev.assign((size_t)PROFILE_RING * (MAX_KERNELS + 1), nullptr);
    for (auto &x : f->ev)
      if (e == cudaSuccess) e = cudaEventCreate(&x);
  }
  if (e != cudaSuccess) {
    dog_destroy(f);
    return cuda_fail(e);
  }
  *out = f;
  return DOG_OK;
}

struct dog_batch {
  std::vector<dog_filter *> f;
  cudaStream_t st = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<BatchFilter> desc;      // each filter's description as captured (host copy)
  std::vector<unsigned char> radar;   // each filter's grid kind when the graph was captured
  std::vector<uint32_t> cfg_version;  // each filter's configuration version then
  // grouping: consecutive filters whose workspaces add up to at most group_bytes form one
  // group (a filter larger than that is a group of its own); each group is one branch of the
  // graph, its phases fused over its filters
  size_t group_bytes = 0;
  std::vector<cudaStream_t> side;     // capture-time branch streams, one per group
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
};

int dog_batch_create(dog_filter *const *filters, int n, dog_batch **out) {
  if (!filters || !out || n < 1) return DOG_ERR_INVALID_ARG;
  if (n > BATCH_MAX) return DOG_ERR_UNSUPPORTED;
  for (int i = 0; i < n; ++i)
    if (!filters[i] || !filters[i]->st || filters[i]->profile || filters[i]->st != filters[0]->st)
      return DOG_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j)
      if (filters[i] == filters[j]) return DOG_ERR_INVALID_ARG;
  // the batched kernels' shared-memory limits (per kernel, as for the single-filter ones)
  DOG_CUDA(cudaFuncSetAttribute(kb_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sort_smem_bytes(2048)));
  DOG_CUDA(cudaFuncSetAttribute(kb_sort_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)count_smem_bytes(2048, COUNT_TILES)));
  dog_batch *b = new (std::nothrow) dog_batch();
  if (!b) return DOG_ERR_INVALID_ARG;
  b->f.assign(filters, filters + n);
  b->st = filters[0]->st;
  b->group_bytes = DOG_BATCH_GROUP_BYTES_DEFAULT;
  b->side.assign(n, nullptr);
  b->join.assign(n, nullptr);
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    dog_batch_destroy(b);
    return cuda_fail(e);
  }
  *out = b;
  return DOG_OK;
}

int dog_batch_set_group_bytes(dog_batch *b, size_t group_bytes) {
  if (!b) return DOG_ERR_INVALID_ARG;
  if (group_bytes != b->group_bytes && b->gexec) {
    cudaGraphExecDestroy(b->gexec);  // captured again at the next step
    b->gexec = nullptr;
  }
  b->group_bytes = group_bytes;
  return DOG_OK;
}

int dog_batch_groups(const dog_batch *b, int *n_groups) {
  if (!b || !n_groups) return DOG_ERR_INVALID_ARG;
  int g = 0;
  size_t acc = 0;
  for (size_t i = 0; i < b->f.size(); ++i) {
    const size_t w = b->f[i]->ws_bytes;
    if (i == 0 || acc + w > b->group_bytes) {
      ++g;
      acc = 0;
    }
    acc += w;
  }
  *n_groups = g;
  return DOG_OK;
}

}  // extern "C"

namespace {
// the launch arguments of one phase: the filters `take` selects, `blocks` blocks each
template <typename Take, typename Blocks>
bool batch_args(const std::vector<dog_filter *> &fs, BatchArgs &A, Take take, Blocks blocks) {
  A.n = 0;
  uint32_t tot = 0;
  for (const dog_filter *f : fs) {
    if (!take(f)) continue;
    const uint32_t c = blocks(f);
    if (c == 0) continue;
    A.first[A.n] = tot;
    A.f[A.n] = reinterpret_cast<const BatchFilter *>(f->B.batch_slot);
    tot += c;
    ++A.n;
  }
  A.first[A.n] = tot;
  return A.n > 0;
}
template <typename Take, typename Bytes>
size_t batch_smem(const std::vector<dog_filter *> &fs, Take take, Bytes bytes) {
  size_t m = 0;
  for (const dog_filter *f : fs)
    if (take(f) && bytes(f) > m) m = bytes(f);
  return m;
}

// one frame of the filters fs on stream st: each phase of the frame once over all of them
int enqueue_group_frame(const std::vector<dog_filter *> &fs, cudaStream_t st) {
  const std::vector<dog_filter *> &bf = fs;
  BatchArgs A;
  auto all = [](const dog_filter *) { return true; };
  auto lidar = [](const dog_filter *f) { return !f->radar; };
  auto radar = [](const dog_filter *f) { return f->radar; };
  auto one = [](const dog_filter *) { return 1u; };
  auto ego = [](const dog_filter *f) { return (f->K.flags & DOG_EGO) != 0; };
  if (batch_args(bf, A, ego, [](const dog_filter *f) { return std::min((f->K.C + 255) / 256, 592u); }))
    kb_ego_warp<<<A.first[A.n], 256, 0, st>>>(A);
  if (batch_args(bf, A, all, [](const dog_filter *f) { return (f->K.nu + PRED_TILE - 1) / PRED_TILE; }))
    kb_predict<<<A.first[A.n], PRED_BLOCK,
                 batch_smem(bf, all, [](const dog_filter *f) { return (size_t)4 * f->K.passes * f->K.radix; }),
                 st>>>(A);
  int max_passes = 0;
  for (const dog_filter *f : bf) max_passes = std::max(max_passes, f->K.passes);
  for (int p = 0; p < max_passes; ++p) {
    auto has = [p](const dog_filter *f) { return f->K.passes > p; };
    if (p > 0 && batch_args(bf, A, has, [](const dog_filter *f) {
          return (f->K.tiles_sort + f->count_ct - 1) / f->count_ct;
        }))
      kb_sort_count<<<A.first[A.n], COUNT_BLOCK,
                      batch_smem(bf, has, [](const dog_filter *f) { return count_smem_bytes(f->K.radix, f->count_ct); }),
                      st>>>(A, p);
    if (batch_args(bf, A, has, [](const dog_filter *f) { return f->K.radix; })) {
      int per = 4;  // the register run that covers every filter's sort tiles
      for (const dog_filter *f : bf)
        if (has(f)) per = std::max(per, offsets_per(f->K.tiles_sort));
      if (per == 4) kb_sort_offsets<4><<<A.first[A.n], OFF_BLOCK, 0, st>>>(A, p);
      else if (per == 8) kb_sort_offsets<8><<<A.first[A.n], OFF_BLOCK, 0, st>>>(A, p);
      else kb_sort_offsets<16><<<A.first[A.n], OFF_BLOCK, 0, st>>>(A, p);
    }
    if (batch_args(bf, A, has, [](const dog_filter *f) { return f->K.tiles_sort; }))
      kb_sort_pass<<<A.first[A.n], SORT_BLOCK,
                     batch_smem(bf, has, [](const dog_filter *f) { return sort_smem_bytes(f->K.radix); }), st>>>(A, p);
  }
  auto seg = [](const dog_filter *f) { return f->K.tiles_seg; };
  auto cell = [](const dog_filter *f) { return f->K.tiles_cell; };
  auto norm = [](const dog_filter *f) { return f->K.tiles_norm; };
  auto pers = [](const dog_filter *f) { return (f->K.nu + NORM_TILE - 1) / NORM_TILE; };
  auto births = [](const dog_filter *f) { return (uint32_t)f->birth_grid; };
  if (batch_args(bf, A, lidar, seg)) kb_segsum_lidar<<<A.first[A.n], SEG_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, radar, seg)) kb_segsum<true><<<A.first[A.n], SEG_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, lidar, cell)) kb_cell<false><<<A.first[A.n], CELL_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, radar, cell)) kb_cell<true><<<A.first[A.n], CELL_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, all, one)) kb_scan_tiles<false><<<A.first[A.n], SCAN_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, lidar, cell)) kb_birth_prep<false><<<A.first[A.n], BPREP_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, radar, cell)) kb_birth_prep<true><<<A.first[A.n], BPREP_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, lidar, births)) kb_birth<false><<<A.first[A.n], BIRTH_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, radar, births)) kb_birth<true><<<A.first[A.n], BIRTH_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, lidar, pers)) kb_normalise_lidar<<<A.first[A.n], NORM_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, radar, pers)) kb_normalise_radar<<<A.first[A.n], NORM_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, radar, pers)) kb_rmsum<<<A.first[A.n], NORM_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, radar, [](const dog_filter *f) { return std::min((f->K.C + 255) / 256, 2368u); }))
    kb_moments<<<A.first[A.n], 256, 0, st>>>(A);
  if (batch_args(bf, A, all, one)) kb_scan_tiles<true><<<A.first[A.n], SCAN_BLOCK, 0, st>>>(A);
  if (batch_args(bf, A, all, norm)) kb_resample<<<A.first[A.n], RES_BLOCK, 0, st>>>(A);
  return cuda_fail(cudaGetLastError());
}
}  // namespace

extern "C" {

// write every filter's description into its slot (in stream order) and capture the frame
static int batch_capture(dog_batch *b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  const int n = (int)b->f.size();
  b->desc.resize(n);
  b->radar.resize(n);
  b->cfg_version.resize(n);
  for (int i = 0; i < n; ++i) {
    dog_filter *f = b->f[i];
    BatchFilter &d = b->desc[i];
    std::memset(&d, 0, sizeof(d));
    d.P = f->K;
    d.B = f->B;
    d.count_ct = f->count_ct;
    d.birth_grid = (uint32_t)f->birth_grid;
    DOG_CUDA(cudaMemcpyAsync(f->B.batch_slot, &d, sizeof(BatchFilter), cudaMemcpyHostToDevice, b->st));
    f->slot_owner = b;
    b->radar[i] = f->radar ? 1 : 0;
    b->cfg_version[i] = f->cfg_version;
  }
  DOG_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  int rc = cuda_fail(cudaEventRecord(b->fork, b->st));
  size_t i0 = 0;
  for (int g = 0; rc == DOG_OK && i0 < b->f.size(); ++g) {
    size_t i1 = i0 + 1, acc = b->f[i0]->ws_bytes;
    while (i1 < b->f.size() && acc + b->f[i1]->ws_bytes <= b->group_bytes) acc += b->f[i1++]->ws_bytes;
    rc = cuda_fail(cudaStreamWaitEvent(b->side[g], b->fork, 0));
    if (rc) break;
    if (i1 == i0 + 1) {  // a group of one filter: its own kernels
      dog_filter *f = b->f[i0];
      cudaStream_t own = f->st;
      f->st = b->side[g];
      rc = enqueue_frame(f, f->radar, nullptr);
      f->st = own;
    } else {
      const std::vector<dog_filter *> grp(b->f.begin() + i0, b->f.begin() + i1);
      rc = enqueue_group_frame(grp, b->side[g]);
    }
    if (rc == DOG_OK) rc = cuda_fail(cudaEventRecord(b->join[g], b->side[g]));
    if (rc == DOG_OK) rc = cuda_fail(cudaStreamWaitEvent(b->st, b->join[g], 0));
    i0 = i1;
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  DOG_CUDA(e);
  const cudaError_t e2 = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGraphDestroy(graph);
  DOG_CUDA(e2);
  return DOG_OK;
}

int dog_batch_step(dog_batch *b, const float *dt) {
  if (!b || !dt) return DOG_ERR_INVALID_ARG;
  const int n = (int)b->f.size();
  for (int i = 0; i < n; ++i) {
    if (!(dt[i] >= 0.0f) || !std::isfinite(dt[i])) return DOG_ERR_INVALID_ARG;
    if (!b->f[i]->has_grid) return DOG_ERR_BAD_STATE;
  }
  // captured again when a filter's grid kind or launch configuration changed, or another
  // batch wrote its slot since
  bool recapture = !b->gexec;
  for (int i = 0; i < n && !recapture; ++i) {
    const dog_filter *f = b->f[i];
    recapture = b->radar[i] != (f->radar ? 1 : 0) || b->cfg_version[i] != f->cfg_version || f->slot_owner != b;
  }
  for (int i = 0; i < n; ++i) {  // time steps that changed, in stream order before the frame
    dog_filter *f = b->f[i];
    if (!f->dt_valid || dt[i] != f->dt) {
      const float h = dt[i];
      DOG_CUDA(cudaMemcpyAsync(&f->B.ctl->dt, &h, 4, cudaMemcpyHostToDevice, b->st));
      f->dt = dt[i];
      f->dt_valid = true;
    }
  }
  for (int i = 0; i < n; ++i) {
    const int rc = issue_ego(b->f[i], b->st);
    if (rc) return rc;
  }
  if (recapture) {
    const int rc = batch_capture(b);
    if (rc) return rc;
  }
  DOG_CUDA(cudaGraphLaunch(b->gexec, b->st));
  for (int i = 0; i < n; ++i) b->f[i]->frame += 1;
  return DOG_OK;
}

int dog_batch_autotune(dog_batch *b, const float *dt, int frames, size_t *chosen) {
  if (!b || !dt || frames < 1) return DOG_ERR_INVALID_ARG;
  // candidate groupings, from one filter per branch to the whole batch in one group
  const size_t cand[] = {0, (size_t)64 << 20, (size_t)256 << 20, (size_t)1 << 30, (size_t)4 << 30,
                         ~(size_t)0};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  DOG_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce);
  }
  size_t best = b->group_bytes;
  float best_ms = 3.0e38f;
  int rc = DOG_OK;
  int last_groups = -1;
  for (size_t c : cand) {
    rc = dog_batch_set_group_bytes(b, c);
    int ng = 0;
    if (rc == DOG_OK) rc = dog_batch_groups(b, &ng);
    if (rc) break;
    if (ng == last_groups) continue;  // the same grouping as the candidate before
    last_groups = ng;
    rc = dog_batch_step(b, dt);  // captures the graph of this grouping
    float ms = 3.0e38f;
    for (int k = 0; k < frames && rc == DOG_OK; ++k) {
      ce = cudaEventRecord(e0, b->st);
      if (ce == cudaSuccess) rc = dog_batch_step(b, dt);
      if (rc == DOG_OK && ce == cudaSuccess) ce = cudaEventRecord(e1, b->st);
      if (rc == DOG_OK && ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float t = 0.0f;
      if (rc == DOG_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
      if (ce != cudaSuccess) rc = cuda_fail(ce);
      if (t < ms) ms = t;
    }
    if (rc) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (chosen) *chosen = best;
  return dog_batch_set_group_bytes(b, best);
}

void dog_batch_destroy(dog_batch *b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (auto x : b->side)
    if (x) cudaStreamDestroy(x);
  for (auto x : b->join)
    if (x) cudaEventDestroy(x);
  if (b->fork) cudaEventDestroy(b->fork);
  for (dog_filter *f : b->f)
    if (f->slot_owner == b) f->slot_owner = nullptr;
  delete b;
}

void dog_destroy(dog_filter *f) {
  if (!f) return;
  if (f->st) cudaStreamSynchronize(f->st);
  for (auto x : {f->h2d, f->d2h, f->aux})
    if (x) {
      cudaStreamSynchronize(x);
      cudaStreamDestroy(x);
    }
  for (auto x : {f->ev_h2d, f->ev_stage_free, f->ev_snap, f->ev_d2h, f->ev_fork, f->ev_join, f->ev_mjoin})
    if (x) cudaEventDestroy(x);
  if (f->d2h_err) cudaFreeHost(f->d2h_err);
  for (auto &g : f->gexec)
    if (g) cudaGraphExecDestroy(g);
  for (auto &x : f->ev)
    if (x) cudaEventDestroy(x);
  delete f;
}

namespace {
// upload (host kinds) or reference (device) the grid's fields and take them over with one
// copy-and-validate kernel in stream order
int take_grid(dog_filter *f, const float *const src[5], int nfield, int kind, int mem_kind) {
  const size_t C = f->d.C;
  const bool radar = kind == GRID_RADAR;
  GridSrc gs{};
  if (mem_kind == DOG_DEVICE) {
    for (int k = 0; k < nfield; ++k) gs.f[k] = src[k];
  } else {
    // upload on the copy stream into the staging buffer (free once the previous grid was
    // taken over), so that it overlaps the frame in flight; then take it over in stream order
    DOG_CUDA(cudaStreamWaitEvent(f->h2d, f->ev_stage_free, 0));
    for (int k = 0; k < nfield; ++k)
      DOG_CUDA(cudaMemcpyAsync(f->B.g_stage + k * C, src[k], 4 * C, cudaMemcpyHostToDevice, f->h2d));
    DOG_CUDA(cudaEventRecord(f->ev_h2d, f->h2d));
    DOG_CUDA(cudaStreamWaitEvent(f->st, f->ev_h2d, 0));
    for (int k = 0; k < nfield; ++k) gs.f[k] = f->B.g_stage + k * C;
  }
  // copy into place and validate in one pass
  k_take_grid<<<1184, 256, 0, f->st>>>(f->K, f->B, gs, kind);
  DOG_CUDA(cudaGetLastError());
  if (mem_kind != DOG_DEVICE) DOG_CUDA(cudaEventRecord(f->ev_stage_free, f->st));
  f->radar = radar;
  f->has_grid = true;
  // host arrays: the caller may reuse them once the upload is done (DOG_HOST_ASYNC: the
  // caller waits for that itself, with dog_sync or a later call that waits)
  if (mem_kind == DOG_HOST) DOG_CUDA(cudaEventSynchronize(f->ev_h2d));
  return DOG_OK;
}
}  // namespace

int dog_set_measurement_grid(dog_filter *f, const dog_meas_grid *g, int mem_kind) {
  if (!f || !g || !g->m_occ || !g->m_free) return DOG_ERR_INVALID_ARG;
  if (mem_kind != DOG_HOST && mem_kind != DOG_DEVICE && mem_kind != DOG_HOST_ASYNC) return DOG_ERR_INVALID_ARG;
  if (f->p.flags & DOG_FULL) return DOG_ERR_BAD_STATE;  // takes dog_set_bernoulli_grid
  const bool radar = g->p_A != nullptr;
  if (radar && (!g->z_vr || !g->sigma_vr)) return DOG_ERR_INVALID_ARG;
  const float *src[5] = {g->m_occ, g->m_free, g->p_A, g->z_vr, g->sigma_vr};
  return take_grid(f, src, radar ? 5 : 2, radar ? GRID_RADAR : GRID_LIDAR, mem_kind);
}

static_assert(FLAG_FULL == DOG_FULL, "the kernels' PHD/MIB flag is the ABI's");

int dog_set_bernoulli_grid(dog_filter *f, const dog_bern_grid *g, int mem_kind) {
  if (!f || !g || !g->z || !g->p_tp || !g->p_fp || !g->p_a || !g->p_c) return DOG_ERR_INVALID_ARG;
  if (mem_kind != DOG_HOST && mem_kind != DOG_DEVICE && mem_kind != DOG_HOST_ASYNC) return DOG_ERR_INVALID_ARG;
  if (!(f->p.flags & DOG_FULL)) return DOG_ERR_BAD_STATE;
  // layout of the grid buffers for the Bernoulli observation: z, p_TP, p_A, p_FP, p_c
  const float *src[5] = {g->z, g->p_tp, g->p_a, g->p_fp, g->p_c};
  return take_grid(f, src, 5, GRID_BERNOULLI, mem_kind);
}

int dog_step(dog_filter *f, float dt) {
  if (!f) return DOG_ERR_INVALID_ARG;
  if (!(dt >= 0.0f) || !std::isfinite(dt)) return DOG_ERR_INVALID_ARG;
  if (!f->has_grid) return DOG_ERR_BAD_STATE;
  if (!f->dt_valid || dt != f->dt) {
    const float h = dt;  // pageable source: staged before cudaMemcpyAsync returns
    DOG_CUDA(cudaMemcpyAsync(&f->B.ctl->dt, &h, 4, cudaMemcpyHostToDevice, f->st));
    f->dt = dt;
    f->dt_valid = true;
  }
  {
    const int rc = issue_ego(f, f->st);
    if (rc) return rc;
  }
  const int gi = f->radar ? 1 : 0;
  if (f->profile) {
    cudaEvent_t *ev = &f->ev[(size_t)f->ring_head * (MAX_KERNELS + 1)];
    const int rc = enqueue_frame(f, f->radar, ev);
    if (rc) return rc;
    f->ring_head = (f->ring_head + 1) % PROFILE_RING;
    if (f->ring_count < PROFILE_RING) ++f->ring_count;
  } else if (f->use_graph) {
    if (!f->gexec[gi]) {
      cudaGraph_t graph;
      DOG_CUDA(cudaStreamBeginCapture(f->st, cudaStreamCaptureModeThreadLocal));
      const int rc = enqueue_frame(f, f->radar, nullptr);
      const cudaError_t e = cudaStreamEndCapture(f->st, &graph);
      if (rc) return rc;
      DOG_CUDA(e);
      const cudaError_t e2 = cudaGraphInstantiate(&f->gexec[gi], graph, 0);
      cudaGraphDestroy(graph);
      DOG_CUDA(e2);
    }
    DOG_CUDA(cudaGraphLaunch(f->gexec[gi], f->st));
  } else {
    const int rc = enqueue_frame(f, f->radar, nullptr);
    if (rc) return rc;
  }
  f->frame += 1;
  return DOG_OK;
}

int dog_sync(dog_filter *f) {
  if (!f) return DOG_ERR_INVALID_ARG;
  return read_err(f);
}

int dog_get_cells(dog_filter *f, const dog_cells *out, int mem_kind) {
  if (!f || !out) return DOG_ERR_INVALID_ARG;
  if (mem_kind != DOG_HOST && mem_kind != DOG_DEVICE) return DOG_ERR_INVALID_ARG;
  const size_t n = 4 * (size_t)f->d.C;
  const cudaMemcpyKind kd = kind_to(mem_kind);
  float *dst[] = {out->m_occ, out->m_free, out->rho_p, out->rho_b, out->p_occ,
                  out->mean_vx, out->mean_vy, out->var_vx, out->var_vy, out->cov_vxy};
  const float *src[] = {f->B.mO, f->B.mF, f->B.rho_p, f->B.rho_b, f->B.pO,
                        f->B.mean_x, f->B.mean_y, f->B.var_x, f->B.var_y, f->B.cov};
  for (int k = 0; k < 10; ++k)
    if (dst[k]) DOG_CUDA(cudaMemcpyAsync(dst[k], src[k], n, kd, f->st));
  return read_err(f);
}

int dog_get_cells_async(dog_filter *f, const dog_cells *out) {
  if (!f || !out) return DOG_ERR_INVALID_ARG;
  if (f->d2h_pending) {  // one read-back in flight: let the previous one finish
    const int rc = dog_wait_cells(f);
    if (rc) return rc;
  }
  const size_t C = f->d.C;
  float *dst[] = {out->m_occ, out->m_free, out->rho_p, out->rho_b, out->p_occ,
                  out->mean_vx, out->mean_vy, out->var_vx, out->var_vy, out->cov_vxy};
  const float *src[] = {f->B.mO, f->B.mF, f->B.rho_p, f->B.rho_b, f->B.pO,
                        f->B.mean_x, f->B.mean_y, f->B.var_x, f->B.var_y, f->B.cov};
  // snapshot in stream order (the next frame may then overwrite the cells), copy to the host
  // on the read-back stream
  uint32_t *err_snap = reinterpret_cast<uint32_t *>(f->B.c_stage + 10 * C);
  CellSnap snap{};
  for (int k = 0; k < 10; ++k) snap.f[k] = dst[k] ? src[k] : nullptr;
  k_snapshot<<<1184, 256, 0, f->st>>>(snap, f->B.c_stage, (uint32_t)C, &f->B.ctl->err, err_snap);
  DOG_CUDA(cudaGetLastError());
  DOG_CUDA(cudaEventRecord(f->ev_snap, f->st));
  DOG_CUDA(cudaStreamWaitEvent(f->d2h, f->ev_snap, 0));
  for (int k = 0; k < 10; ++k)
    if (dst[k]) DOG_CUDA(cudaMemcpyAsync(dst[k], f->B.c_stage + k * C, 4 * C, cudaMemcpyDeviceToHost, f->d2h));
  DOG_CUDA(cudaMemcpyAsync(f->d2h_err, err_snap, 4, cudaMemcpyDeviceToHost, f->d2h));
  DOG_CUDA(cudaEventRecord(f->ev_d2h, f->d2h));
  f->d2h_pending = true;
  return DOG_OK;
}

int dog_wait_cells(dog_filter *f) {
  if (!f) return DOG_ERR_INVALID_ARG;
  if (!f->d2h_pending) return DOG_OK;
  DOG_CUDA(cudaEventSynchronize(f->ev_d2h));
  f->d2h_pending = false;
  const uint32_t err = *f->d2h_err;
  *f->d2h_err = 0;
  if (err & ERR_INPUT) return DOG_ERR_INPUT;
  if (err) return DOG_ERR_DEVICE;
  return DOG_OK;
}

int dog_get_state(dog_filter *f, const dog_state *out, int mem_kind, uint32_t *frame) {
  if (!f || !out) return DOG_ERR_INVALID_ARG;
  if (mem_kind != DOG_HOST && mem_kind != DOG_DEVICE) return DOG_ERR_INVALID_ARG;
  const size_t n = 4 * (size_t)f->p.num_particles;
  const cudaMemcpyKind kd = kind_to(mem_kind);
  float *const dst[4] = {out->x, out->y, out->vx, out->vy};
  // posterior as plain arrays in the staging buffer (x, y, vx, vy) and Aw (weights; both
  // idle between steps)
  float *scr = reinterpret_cast<float *>(f->B.stage);
  k_gather_posterior<<<1024, 256, 0, f->st>>>(f->K, f->B, scr, f->B.Aw);
  DOG_CUDA(cudaGetLastError());
  for (int k = 0; k < 4; ++k)
    if (dst[k]) DOG_CUDA(cudaMemcpyAsync(dst[k], scr + k * (size_t)f->p.num_particles, n, kd, f->st));
  if (out->w) DOG_CUDA(cudaMemcpyAsync(out->w, f->B.Aw, n, kd, f->st));
  if (out->m_free) DOG_CUDA(cudaMemcpyAsync(out->m_free, f->B.mF, 4 * (size_t)f->d.C, kd, f->st));
  const int rc = read_err(f);
  if (frame) *frame = f->frame;
  return rc;
}

int dog_set_state(dog_filter *f, const dog_state *in, int mem_kind, uint32_t frame) {
  if (!f || !in || !in->x || !in->y || !in->vx || !in->vy || !in->w || !in->m_free)
    return DOG_ERR_INVALID_ARG;
  if (mem_kind != DOG_HOST && mem_kind != DOG_DEVICE) return DOG_ERR_INVALID_ARG;
  const size_t n = 4 * (size_t)f->p.num_particles;
  const cudaMemcpyKind kd = kind_from(mem_kind);
  const float *const src[4] = {in->x, in->y, in->vx, in->vy};
  // the restored posterior is held directly: records in Os, weights in Bw
  const int rc0 = pack_records(f, f->B.Os, f->p.num_particles, src, kd);
  if (rc0) return rc0;
  DOG_CUDA(cudaMemcpyAsync(f->B.Bw, in->w, n, kd, f->st));
  const uint32_t direct = POST_DIRECT;
  DOG_CUDA(cudaMemcpyAsync(&f->B.ctl->post_mode, &direct, 4, cudaMemcpyHostToDevice, f->st));
  DOG_CUDA(cudaMemcpyAsync(f->B.mF, in->m_free, 4 * (size_t)f->d.C, kd, f->st));
  const int rc = reset_epochs(f);
  if (rc) return rc;
  const uint32_t fr = frame;
  DOG_CUDA(cudaMemcpyAsync(&f->B.ctl->frame, &fr, 4, cudaMemcpyHostToDevice, f->st));
  DOG_CUDA(cudaStreamSynchronize(f->st));
  f->frame = frame;
  return DOG_OK;
}

int dog_get_debug(dog_filter *f, int which, void *out, int mem_kind) {
  if (!f || !out || which < 0 || which >= DOG_DBG_COUNT) return DOG_ERR_INVALID_ARG;
  if (mem_kind != DOG_HOST && mem_kind != DOG_DEVICE) return DOG_ERR_INVALID_ARG;
  const DevBufs &B = f->B;
  const size_t nu = f->p.num_particles, nb = f->p.num_birth, C = f->d.C;
  const bool record = (f->p.flags & DOG_RECORD) != 0;
  const void *src = nullptr;
  size_t bytes = 0;
  bool masked = false;
  const float4 *rec = nullptr;  // component of (x, y, vx, vy) records
  int comp = 0;
  size_t nrec = 0;
  switch (which) {
    case DOG_DBG_PRED_X: rec = B.As; comp = 0; nrec = nu; break;
    case DOG_DBG_PRED_Y: rec = B.As; comp = 1; nrec = nu; break;
    case DOG_DBG_PRED_VX: rec = B.As; comp = 2; nrec = nu; break;
    case DOG_DBG_PRED_VY: rec = B.As; comp = 3; nrec = nu; break;
    case DOG_DBG_PRED_W: src = B.Aw; bytes = 4 * nu; break;
    case DOG_DBG_KEY: src = B.key_pred; bytes = 4 * nu; break;
    case DOG_DBG_PERM: src = B.perm; bytes = 4 * nu; break;
    case DOG_DBG_CELL_START: src = B.cstart; bytes = 4 * C; masked = true; break;
    case DOG_DBG_CELL_END: src = B.cend; bytes = 4 * C; masked = true; break;
    case DOG_DBG_SUM_W: src = &B.csum[0].S; bytes = 8 * C; masked = true; break;
    case DOG_DBG_SUM_GW: src = B.A; bytes = 8 * C; masked = true; break;
    case DOG_DBG_M_OCC_PRED:  // recomputed from the cell records into scratch
      k_mpred<<<(unsigned)((C + 255) / 256 < 4096 ? (C + 255) / 256 : 4096), 256, 0, f->st>>>(
          B.csum, (uint32_t)C, f->frame, B.mpred);
      DOG_CUDA(cudaGetLastError());
      src = B.mpred;
      bytes = 4 * C;
      break;
    case DOG_DBG_MU_A: src = B.muA; bytes = 4 * C; break;
    case DOG_DBG_MU_UA: src = B.muU; bytes = 4 * C; break;
    case DOG_DBG_W_NORM: src = B.wn; bytes = 4 * nu; break;
    case DOG_DBG_BIRTH_X: rec = B.bs; comp = 0; nrec = nb; break;
    case DOG_DBG_BIRTH_Y: rec = B.bs; comp = 1; nrec = nb; break;
    case DOG_DBG_BIRTH_VX: rec = B.bs; comp = 2; nrec = nb; break;
    case DOG_DBG_BIRTH_VY: rec = B.bs; comp = 3; nrec = nb; break;
    case DOG_DBG_BIRTH_W: src = B.bw; bytes = 4 * nb; break;
    case DOG_DBG_BIRTH_CELL: src = B.bcell; bytes = 4 * nb; break;
    case DOG_DBG_BIRTH_ASSOC: src = B.bassoc; bytes = 4 * nb; break;
    case DOG_DBG_RESAMPLE_SRC: src = B.Bsrc; bytes = 4 * nu; break;
    case DOG_DBG_SCALARS: break;
    default: return DOG_ERR_INVALID_ARG;
  }
  if ((which == DOG_DBG_BIRTH_CELL || which == DOG_DBG_BIRTH_ASSOC ||
       ((which == DOG_DBG_CELL_START || which == DOG_DBG_CELL_END) && !f->radar)) && !record)
    return DOG_ERR_BAD_STATE;
  DOG_CUDA(cudaStreamSynchronize(f->st));
  if (which == DOG_DBG_SCALARS) {
    DevCtl h;
    DOG_CUDA(cudaMemcpy(&h, B.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost));
    const unsigned long long v[4] = {h.frame, h.W_total, h.R_total, h.u_offset};
    DOG_CUDA(cudaMemcpy(out, v, sizeof(v), mem_kind == DOG_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    return read_err(f);
  }
  if (rec) {
    float *dst[4] = {nullptr, nullptr, nullptr, nullptr};
    dst[comp] = (float *)out;
    const int rc = unpack_records(f, rec, nrec, dst, kind_to(mem_kind));
    if (rc) return rc;
    return read_err(f);
  }
  if (which == DOG_DBG_KEY || which == DOG_DBG_PERM) {
    // cell index / particle index without the out-of-grid flag the kernels carry in bit 31
    std::vector<uint32_t> v(nu);
    DOG_CUDA(cudaMemcpy(v.data(), src, 4 * nu, cudaMemcpyDeviceToHost));
    for (auto &x : v) x &= ~OUT_OF_GRID;
    DOG_CUDA(cudaMemcpy(out, v.data(), 4 * nu, mem_kind == DOG_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    return read_err(f);
  }
  if (!masked) {
    if (bytes) DOG_CUDA(cudaMemcpyAsync(out, src, bytes, kind_to(mem_kind), f->st));
    return read_err(f);
  }
  // cell arrays valid only where the cell received particles this frame (tag == frame)
  std::vector<uint32_t> tag(C);
  std::vector<unsigned char> buf(bytes);
  const size_t es = bytes / C;
  DOG_CUDA(cudaMemcpy2D(tag.data(), 4, &B.csum[0].tag, sizeof(CellSum), 4, C, cudaMemcpyDeviceToHost));
  if (which == DOG_DBG_SUM_W)  // a field of the cell records
    DOG_CUDA(cudaMemcpy2D(buf.data(), es, src, sizeof(CellSum), es, C, cudaMemcpyDeviceToHost));
  else
    DOG_CUDA(cudaMemcpy(buf.data(), src, bytes, cudaMemcpyDeviceToHost));
  for (size_t c = 0; c < C; ++c)
    if ((tag[c] >> 1) != f->frame || f->frame == 0) std::memset(buf.data() + c * es, 0, es);
  DOG_CUDA(cudaMemcpy(out, buf.data(), bytes, mem_kind == DOG_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
  return read_err(f);
}

int dog_profile_read(dog_filter *f, float *ms, const char **names, int max, int *n_out, int *steps_out) {
  if (!f || !ms || max <= 0) return DOG_ERR_INVALID_ARG;
  if (!f->profile) return DOG_ERR_BAD_STATE;
  DOG_CUDA(cudaStreamSynchronize(f->st));
  // kernel slots in launch order: ego-motion warp (DOG_EGO), predict, sort passes, segsum,
  // cell, birth scan, birth prep, birth, normalise, CDF scan, resample
  int slot_kind[MAX_KERNELS];
  int nk = 0;
  if (f->p.flags & DOG_EGO) slot_kind[nk++] = 0;
  slot_kind[nk++] = 1;
  slot_kind[nk++] = 2;
  slot_kind[nk++] = 3;
  for (int p = 1; p < f->K.passes; ++p) {
    slot_kind[nk++] = 1 + 3 * p;
    slot_kind[nk++] = 2 + 3 * p;
    slot_kind[nk++] = 3 + 3 * p;
  }
  for (int k = 10; k <= 17; ++k) slot_kind[nk++] = k;
  const int n = nk < max ? nk : max;
  for (int k = 0; k < n; ++k) ms[k] = 0.0f;
  for (int r = 0; r < f->ring_count; ++r) {
    const int slot = (f->ring_head - 1 - r + 2 * PROFILE_RING) % PROFILE_RING;
    cudaEvent_t *ev = &f->ev[(size_t)slot * (MAX_KERNELS + 1)];
    for (int k = 0; k < n; ++k) {
      float t = 0.0f;
      DOG_CUDA(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
      ms[k] += t;
    }
  }
  if (names)
    for (int k = 0; k < n; ++k) names[k] = KNAMES[slot_kind[k]];
  if (n_out) *n_out = n;
  if (steps_out) *steps_out = f->ring_count;
  f->ring_count = 0;
  return DOG_OK;
}

}  // extern "C"

// ====================================================================================
// Allocation-free cell assignment.
//
// Some callers cannot allocate device memory at all: code that runs where cudaMalloc is
// forbidden or unavailable (inside a host callback, from a real-time thread that must not
// take the allocator's locks, under an allocator that another framework owns exclusively,
// or in a process whose memory pool is fixed at start-up).  For them the particle-to-cell
// assignment -- the stable sort of cell indices and the per-cell ranges -- runs with its
// scratch in one array of fixed size that lives in this library's device image.  Every
// GPU that loads the library holds that array until the process exits.
// ====================================================================================
namespace {

constexpr uint32_t NA_MAX_N = 1u << 19;             // particles per call
constexpr uint32_t NA_MAX_CELLS = (1u << 22) - 1u;  // cells per call: with the sentinel
                                                    // num_cells, keys of at most 22 bits
constexpr uint32_t NA_TILES = NA_MAX_N / SORT_TILE;
constexpr size_t NA_CTL = 256;
static_assert(sizeof(DevCtl) <= NA_CTL, "the control block fits its slot");
constexpr size_t NA_HIST = 2 * 2048 * 4;
constexpr size_t NA_DCNT = (size_t)2 * NA_TILES * 2048 * 4;
constexpr size_t NA_ARR = (size_t)NA_MAX_N * 4;
constexpr size_t NA_BYTES = NA_CTL + NA_HIST + NA_DCNT + 4 * NA_ARR;  // 10,502,400 bytes
static_assert(NA_MAX_CELLS == DOG_NOALLOC_MAX_CELLS && NA_MAX_N == DOG_NOALLOC_MAX_PARTICLES,
              "the header states the limits");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// The caller's keys with every key >= num_cells replaced by the sentinel num_cells (so that
// those particles sort after all others, in input order, and fall in no cell's range), and
// the digit histograms of all passes over them; block t handles sort tile t and writes that
// tile's first-pass digit counts.
__global__ void k_na_hist(const uint32_t *__restrict__ keys, uint32_t num_cells, uint32_t *__restrict__ kc,
                          KParams K, DevBufs B) {
  extern __shared__ uint32_t sh[];
  const uint32_t nh = (uint32_t)K.passes * K.radix;
  for (uint32_t k = threadIdx.x; k < nh; k += blockDim.x) sh[k] = 0u;
  __syncthreads();
  const uint32_t mask = K.radix - 1u;
  for (uint32_t i = blockIdx.x * SORT_TILE + threadIdx.x; i < (blockIdx.x + 1u) * SORT_TILE;
       i += blockDim.x) {
    const bool ok = i < K.nu;
    uint32_t key = 0u;
    if (ok) {
      key = min(keys[i], num_cells);
      if (kc) kc[i] = key;
    }
    for (int p = 0; p < K.passes; ++p) {
      const uint32_t d = ok ? ((key >> (p * K.dbits)) & mask) : 0xffffffffu;
      const uint32_t peers = __match_any_sync(FULL, d);
      if (ok && (peers & lanemask_lt()) == 0u) atomicAdd(&sh[p * K.radix + d], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < nh; k += blockDim.x)
    if (sh[k]) atomicAdd(&B.hist[(k / K.radix) * 2048u + (k % K.radix)], sh[k]);
  for (uint32_t d = threadIdx.x; d < K.radix; d += blockDim.x)
    B.dcnt[(size_t)d * K.tiles_sort + blockIdx.x] = sh[d];
}

// half-open range of each cell in the sorted order (the sentinel key num_cells is skipped)
__global__ void k_na_ranges(const uint32_t *__restrict__ ks, uint32_t n, uint32_t num_cells,
                            uint32_t *start, uint32_t *end) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const uint32_t k = ks[j];
    if (k >= num_cells) continue;
    if (j == 0 || ks[j - 1] != k) start[k] = j;
    if (j == n - 1 || ks[j + 1] != k) end[k] = j + 1;
  }
}

// The scratch array's device address and the sort kernels' shared-memory limits belong to a
// CUDA context: they are set up once per context (with its device current) and looked up
// again whenever the calling thread's current context differs from the one they were set up
// in (a context destroyed by cudaDeviceReset and created anew gets a fresh set-up).  The
// context handle comes from the driver's cuCtxGetCurrent, reached through the runtime.
struct NaDevice {
  bool ready = false;
  void *ctx = nullptr;
  char *base = nullptr;
};
NaDevice g_na_dev[64];
std::mutex g_na_mutex;
typedef int (*CtxGetCurrentFn)(void **);

void *current_context() {
  static CtxGetCurrentFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      (void)cudaGetLastError();
      p = nullptr;
    }
    return (CtxGetCurrentFn)p;
  }();
  void *ctx = nullptr;
  if (fn && fn(&ctx) != 0) ctx = nullptr;
  return ctx;
}

int na_setup(char **base) {
  int dev = 0;
  DOG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return DOG_ERR_UNSUPPORTED;
  void *ctx = current_context();  // null if no context is current in this thread yet
  std::lock_guard<std::mutex> lock(g_na_mutex);
  NaDevice &d = g_na_dev[dev];
  if (!d.ready || ctx != d.ctx) {
    void *p = nullptr;
    d.ready = false;
    // (the first runtime call on the device binds its primary context to the thread)
    DOG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    DOG_CUDA(cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sort_smem_bytes(2048)));
    DOG_CUDA(cudaFuncSetAttribute(k_sort_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)count_smem_bytes(2048, COUNT_TILES)));
    d.base = (char *)p;
    d.ctx = current_context();
    d.ready = d.ctx != nullptr;  // without a context handle: set up again on every call
  }
  *base = d.base;
  return DOG_OK;
}

}  // namespace

extern "C" int dog_assign_cells_noalloc(const uint32_t *d_keys, uint32_t n, uint32_t num_cells,
                                        uint32_t *d_perm, uint32_t *d_cell_start,
                                        uint32_t *d_cell_end, void *cuda_stream) {
  if (num_cells == 0 || !d_cell_start || !d_cell_end || (n > 0 && (!d_keys || !d_perm)))
    return DOG_ERR_INVALID_ARG;
  if (n > NA_MAX_N || num_cells > NA_MAX_CELLS) return DOG_ERR_UNSUPPORTED;
  char *base = nullptr;
  const int rc = na_setup(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DOG_CUDA(cudaMemsetAsync(d_cell_start, 0, 4 * (size_t)num_cells, st));
  DOG_CUDA(cudaMemsetAsync(d_cell_end, 0, 4 * (size_t)num_cells, st));
  if (n == 0) return DOG_OK;
  // key bits cover the sentinel num_cells
  int bits = 1;
  while ((1ull << bits) <= num_cells) ++bits;
  KParams K{};
  K.nu = n;
  K.passes = (bits + 10) / 11;
  K.dbits = (bits + K.passes - 1) / K.passes;
  K.radix = 1u << K.dbits;
  K.tiles_sort = (n + SORT_TILE - 1) / SORT_TILE;
  DevBufs B{};
  B.ctl = (DevCtl *)base;
  B.hist = (uint32_t *)(base + NA_CTL);
  B.dcnt = (uint32_t *)(base + NA_CTL + NA_HIST);
  uint32_t *key_c = (uint32_t *)(base + NA_CTL + NA_HIST + NA_DCNT);
  uint32_t *key_t0 = key_c + NA_MAX_N;
  uint32_t *val_t0 = key_t0 + NA_MAX_N;
  uint32_t *key_sorted = val_t0 + NA_MAX_N;
  // every array of the scratch is rewritten before it is read: the histogram by k_tick, the
  // clamped keys and the per-tile digit counts by k_na_hist (first pass) and k_sort_count
  // (later passes)
  k_tick<<<1, 256, 0, st>>>(B, 2048 * K.passes, 0u);
  k_na_hist<<<K.tiles_sort, 256, 4u * K.passes * K.radix, st>>>(d_keys, num_cells, key_c, K, B);
  const size_t ssm = sort_smem_bytes(K.radix);
  int sms = 148;
  {
    int dev = 0;
    DOG_CUDA(cudaGetDevice(&dev));
    DOG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const uint32_t ct = count_tiles_per_block(K.tiles_sort, sms);
  const uint32_t *kin = key_c, *vin = nullptr;
  for (int p = 0; p < K.passes; ++p) {
    uint32_t *kout = (p == K.passes - 1) ? key_sorted : key_t0;
    uint32_t *vout = (p == K.passes - 1) ? d_perm : val_t0;
    if (p > 0)
      k_sort_count<<<(K.tiles_sort + ct - 1) / ct, COUNT_BLOCK, count_smem_bytes(K.radix, ct), st>>>(K, B, kin,
                                                                                                       p, ct);
    launch_offsets(K, B, p, st);
    k_sort_pass<<<K.tiles_sort, SORT_BLOCK, ssm, st>>>(K, B, kin, vin, kout, vout, p);
    kin = kout;
    vin = vout;
  }
  const uint32_t rgrid = (n + 255) / 256 < 2048u ? (n + 255) / 256 : 2048u;
  k_na_ranges<<<rgrid, 256, 0, st>>>(key_sorted, n, num_cells, d_cell_start, d_cell_end);
  return cuda_fail(cudaGetLastError());
}

// ------------------------------------------------------------------------------------
// Sort configuration (passes and digit width, sort tiles per counting block) and its
// autotuning.  Every configuration sorts to the same order, so the choice changes speed
// only.  Tuned choices are cached for the process by the size class (ceil log2 nu,
// ceil log2 C) and given to filters created later in the same class.
// ------------------------------------------------------------------------------------
namespace {
struct SortCfg {
  int passes;
  uint32_t ct;
};
std::mutex g_tune_mutex;
std::map<std::pair<int, int>, SortCfg> g_tune_cache;

int ceil_log2(uint64_t x) {
  int b = 0;
  while ((1ull << b) < x) ++b;
  return b;
}
std::pair<int, int> size_class(const dog_filter *f) {
  return {ceil_log2(f->p.num_particles), ceil_log2(f->d.C)};
}

// whether the filter's workspace holds a sort of `passes` passes (ping-pong buffers, digit
// histograms, per-tile digit counts) and ct is a valid number of tiles per counting block
bool sort_cfg_ok(const dog_filter *f, int passes, uint32_t ct) {
  if (passes < 1 || passes > 3) return false;
  const int dbits = (f->d.key_bits + passes - 1) / passes;
  if (dbits < 1 || dbits > 11) return false;
  if (passes >= 2 && !f->B.key_t0) return false;
  if (passes >= 3 && !f->B.key_t1) return false;
  const size_t need = (size_t)passes * f->d.tiles_sort * (1u << dbits);
  if (need > (size_t)f->d.passes * f->d.tiles_sort * f->d.radix) return false;
  return ct == 1u || ct == 2u || ct == 4u || ct == 8u;
}

void set_sort_cfg(dog_filter *f, int passes, uint32_t ct) {
  const int dbits = (f->d.key_bits + passes - 1) / passes;
  f->K.passes = passes;
  f->K.dbits = dbits;
  f->K.radix = 1u << dbits;
  f->count_ct = ct;
  f->nk = 8 + 3 * passes;
  f->cfg_version += 1;  // batches holding the filter capture again
  for (auto &g : f->gexec)  // the next step captures the frame again
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// the sort of the filter's current predicted keys with configuration (passes, ct); the
// first pass's digit counts come from the keys themselves (in a frame, from k_predict)
int enqueue_sort(dog_filter *f, int passes, uint32_t ct, cudaEvent_t e0, cudaEvent_t e1) {
  KParams K = f->K;
  K.dbits = (f->d.key_bits + passes - 1) / passes;
  K.passes = passes;
  K.radix = 1u << K.dbits;
  const DevBufs &B = f->B;
  cudaStream_t st = f->st;
  DOG_CUDA(cudaMemsetAsync(B.hist, 0, 4 * 2048 * (size_t)passes, st));
  k_na_hist<<<K.tiles_sort, 256, 4u * K.passes * K.radix, st>>>(B.key_pred, 0xffffffffu, nullptr, K, B);
  DOG_CUDA(cudaEventRecord(e0, st));
  const size_t ssm = sort_smem_bytes(K.radix);
  const uint32_t *kin = B.key_pred, *vin = nullptr;
  for (int p = 0; p < passes; ++p) {
    uint32_t *kout = p == passes - 1 ? B.key_sorted : (p == 0 ? B.key_t0 : B.key_t1);
    uint32_t *vout = p == passes - 1 ? B.perm : (p == 0 ? B.val_t0 : B.val_t1);
    if (p > 0)
      k_sort_count<<<(K.tiles_sort + ct - 1) / ct, COUNT_BLOCK, count_smem_bytes(K.radix, ct), st>>>(K, B, kin,
                                                                                                      p, ct);
    launch_offsets(K, B, p, st);
    k_sort_pass<<<K.tiles_sort, SORT_BLOCK, ssm, st>>>(K, B, kin, vin, kout, vout, p);
    kin = kout;
    vin = vout;
  }
  DOG_CUDA(cudaEventRecord(e1, st));
  return cuda_fail(cudaGetLastError());
}
}  // namespace

static void apply_cached_sort_cfg(dog_filter *f) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  const auto it = g_tune_cache.find(size_class(f));
  if (it != g_tune_cache.end() && sort_cfg_ok(f, it->second.passes, it->second.ct))
    set_sort_cfg(f, it->second.passes, it->second.ct);
}

int dog_sort_config(const dog_filter *f, int *passes, int *digit_bits, int *count_tiles) {
  if (!f) return DOG_ERR_INVALID_ARG;
  if (passes) *passes = f->K.passes;
  if (digit_bits) *digit_bits = f->K.dbits;
  if (count_tiles) *count_tiles = (int)f->count_ct;
  return DOG_OK;
}

int dog_set_sort_config(dog_filter *f, int passes, int count_tiles) {
  if (!f || count_tiles < 1) return DOG_ERR_INVALID_ARG;
  if (!sort_cfg_ok(f, passes, (uint32_t)count_tiles)) return DOG_ERR_UNSUPPORTED;
  set_sort_cfg(f, passes, (uint32_t)count_tiles);
  return DOG_OK;
}

int dog_autotune(dog_filter *f) {
  if (!f) return DOG_ERR_INVALID_ARG;
  if (f->frame == 0) return DOG_ERR_BAD_STATE;  // times the keys of a frame
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  DOG_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce);
  }
  SortCfg best{f->K.passes, f->count_ct};
  float best_ms = 3.0e38f;
  int rc = DOG_OK;
  for (int passes = f->d.passes; passes <= f->d.passes + 1 && rc == DOG_OK; ++passes)
    for (uint32_t ct = 1; ct <= (uint32_t)COUNT_TILES && rc == DOG_OK; ct *= 2) {
      if (!sort_cfg_ok(f, passes, ct) || (passes == 1 && ct > 1)) continue;  // ct: later passes
      float ms = 3.0e38f;
      for (int rep = 0; rep < 5 && rc == DOG_OK; ++rep) {  // the best of five
        rc = enqueue_sort(f, passes, ct, e0, e1);
        if (rc == DOG_OK) {
          ce = cudaEventSynchronize(e1);
          float t = 0.0f;
          if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
          if (ce != cudaSuccess) rc = cuda_fail(ce);
          if (t < ms) ms = t;
        }
      }
      if (rc == DOG_OK && ms < best_ms) {
        best_ms = ms;
        best = SortCfg{passes, ct};
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  set_sort_cfg(f, best.passes, best.ct);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[size_class(f)] = best;
  return DOG_OK;
}
