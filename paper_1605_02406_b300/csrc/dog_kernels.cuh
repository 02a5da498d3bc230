// dog_kernels.cuh -- the per-frame kernels of the DS-PHD/MIB filter (Sect. VII, Alg. 1-7).
//
// Frame data flow (nu persistent particles, nu_b newborn slots, C cells):
//   k_predict     Alg. 1  B -> A: constant-velocity prediction with Philox process noise,
//                          persistence weight, cell index; digit histograms for the sort
//   k_sort_count / k_sort_offsets / k_sort_pass
//                 Alg. 2  LSD radix passes of (cell index, particle index), reduce-then-scan
//   k_segsum      Alg. 2/3 cell ranges and exact fixed-point per-cell sums of w (and g w)
//   k_cell        Alg. 3  occupancy prediction, DS update, newborn split, normalisers;
//                          per-tile lists of cells with newborn mass
//   k_scan_tiles          prefix of the tiles' newborn masses
//   k_birth_prep  Alg. 5  slot range, associated share and weights of each birth cell
//   k_birth       Alg. 5  newborn particles, slots proportional to the newborn mass
//   k_normalise   Alg. 4  normalised persistent weights, tile sums of the joint weights
//                          (the lidar filter's velocity moments were summed in k_segsum_lidar)
//   k_rmsum / k_moments  Alg. 6  (radar filter) the cells' velocity moments from w'
//   k_scan_tiles          CDF of the joint weights over tiles; the frame counter advanced
//   k_resample    Alg. 7  systematic resampling A + newborns -> B
// What a frame accumulates into is cleared by its last reader within the frame (each sort
// pass its digit histogram, the CDF scan the joint-weight tile sums), so a frame needs no
// separate start-of-frame kernel.
// No block waits for another block of the same launch: every cross-block dependency is a
// kernel boundary.
#pragma once
#include "dog_common.cuh"
#include "dog_math.cuh"

namespace dog {

// ====================================================================================
// k_tick: reset of the digit histograms and the joint-weight tile sums, and the frame
// counter advanced.  A filter's frames need no tick: each sort pass clears its digit
// histogram once the offsets are taken from it, and the CDF scan clears the tile sums it
// reads and advances the counter (this_frame).  The allocation-free sort starts with one.
// ====================================================================================
__device__ __forceinline__ void tick_body(const DevBufs &B, int n_hist, uint32_t n_cdf) {
  for (int i = threadIdx.x; i < n_hist; i += blockDim.x) B.hist[i] = 0u;
  // the joint-weight sums of the resampling tiles, which the normalisation (persistent
  // sources) and the newborn kernel (newborn slots) add into
  for (uint32_t i = threadIdx.x; i < n_cdf; i += blockDim.x) B.cdf_tile[i] = 0ull;
  if (threadIdx.x == 0) B.ctl->frame += 1u;
}
__global__ void k_tick(DevBufs B, int n_hist, uint32_t n_cdf) { tick_body(B, n_hist, n_cdf); }

// ====================================================================================
// k_init: initial state -- particles uniform over the grid, birth-distribution
// velocities, weight 0 (frame 0 draws); free mass 0.
// ====================================================================================
__global__ void k_init(KParams P, DevBufs B) {
  const uint32_t stride = gridDim.x * blockDim.x;
  const float gx = __fmul_rn((float)P.W, P.s), gy = __fmul_rn((float)P.H, P.s);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P.nu; i += stride) {
    const U4 r = philox(i, 0u, TAG_INIT, P.seed_lo, P.seed_hi);
    float n0, n1;
    gauss2(r.c, r.d, n0, n1);
    B.Os[i] = make_float4(__fmul_rn(u01_co(r.a), gx), __fmul_rn(u01_co(r.b), gy),
                          __fmul_rn(P.sigma_B, n0), __fmul_rn(P.sigma_B, n1));
    B.Bw[i] = 0.0f;
  }
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < P.C; c += stride) B.mF[c] = 0.0f;
  if (blockIdx.x == 0 && threadIdx.x == 0) B.ctl->post_mode = POST_DIRECT;
}

// posterior particle i (record and weight) under either post_mode
__device__ __forceinline__ float4 posterior_record(const KParams &P, const DevBufs &B, uint32_t mode,
                                                   uint32_t i) {
  if (mode == POST_DIRECT) return __ldg(B.Os + i);
  const uint32_t j = __ldg(B.Bsrc + i);
  return j < P.nu ? __ldg(B.Os + j) : __ldg(B.bs + (j - P.nu));
}

// posterior state as plain arrays: out[0..3][i] = x, y, vx, vy and w[i] (checkpoints)
__global__ void k_gather_posterior(KParams P, DevBufs B, float *__restrict__ out, float *__restrict__ w) {
  const uint32_t mode = B.ctl->post_mode;
  const float wn = B.ctl->w_new;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P.nu; i += gridDim.x * blockDim.x) {
    const float4 r = posterior_record(P, B, mode, i);
    out[i] = r.x;
    out[P.nu + i] = r.y;
    out[2 * (size_t)P.nu + i] = r.z;
    out[3 * (size_t)P.nu + i] = r.w;
    w[i] = mode == POST_DIRECT ? B.Bw[i] : wn;
  }
}

// ====================================================================================
// record <-> plain arrays (state checkpoint and diagnostics; not on the per-frame path)
// ====================================================================================
__global__ void k_unpack(const float4 *__restrict__ rec, uint32_t n, float *__restrict__ out /* [4][n] */) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 r = rec[i];
    out[i] = r.x;
    out[n + i] = r.y;
    out[2 * (size_t)n + i] = r.z;
    out[3 * (size_t)n + i] = r.w;
  }
}
__global__ void k_pack(const float *__restrict__ in /* [4][n] */, uint32_t n, float4 *__restrict__ rec) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    rec[i] = make_float4(in[i], in[n + i], in[2 * (size_t)n + i], in[3 * (size_t)n + i]);
}

// snapshot for an asynchronous read-back: the requested cell fields (null = skipped) into
// the read-back staging buffer, and the error word (then cleared), in one launch
struct CellSnap {
  const float *f[10];
};

__global__ void k_snapshot(CellSnap src, float *__restrict__ stage, uint32_t C, uint32_t *err,
                           uint32_t *err_snap) {
  const uint32_t stride = gridDim.x * blockDim.x;
  // 16-byte accesses when every row starts on a 16-byte boundary (the cell arrays do; C % 4)
  const bool vec = (C & 3u) == 0u;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    if (!src.f[k]) continue;  // uniform
    if (vec) {
      const float4 *in = reinterpret_cast<const float4 *>(src.f[k]);
      float4 *out = reinterpret_cast<float4 *>(stage + (size_t)k * C);
      for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C / 4u; c += stride) out[c] = __ldg(in + c);
    } else {
      for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += stride)
        stage[(size_t)k * C + c] = __ldg(src.f[k] + c);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *err_snap = *err;
    *err = 0u;
  }
}

// predicted occupied mass m_pred = min(S, 1) of every cell for the diagnostic read, from
// the cell records (S and the frame tag) exactly as k_cell computes it; 0 where the cell
// received no particle this frame
__global__ void k_mpred(const CellSum *__restrict__ cs, uint32_t C, uint32_t frame, float *__restrict__ out) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    const bool occ = frame != 0u && (cs[c].tag >> 1) == frame;
    out[c] = occ ? fminf(fx40_to_f(cs[c].S), 1.0f) : 0.0f;
  }
}

// ====================================================================================
// the measurement grid of the next frame: copied into place from the staging buffer or the
// caller's device arrays and validated in the same pass (m_O, m_F in [0, 1] with sum <= 1;
// radar: p_A in [0, 1], sigma_vr > 0 where p_A > 0, z_vr finite); a violation latches
// ERR_INPUT
// ====================================================================================
struct GridSrc {
  const float *f[5];  // m_occ, m_free, p_A, z_vr, sigma_vr (the last three: radar only)
};

enum : int { GRID_LIDAR = 0, GRID_RADAR = 1, GRID_BERNOULLI = 2 };

__global__ void k_take_grid(KParams P, DevBufs B, GridSrc src, int kind) {
  const uint32_t stride = gridDim.x * blockDim.x;
  bool bad = false;
  // lidar grids on 16-byte boundaries (the staging buffer always; a caller's device arrays
  // usually): four cells per thread and access
  bool vec = kind == GRID_LIDAR && (P.C & 3u) == 0u;
  for (int k = 0; k < 2; ++k) vec = vec && (reinterpret_cast<uintptr_t>(src.f[k]) & 15u) == 0u;
  if (vec) {
    const float4 *o4 = reinterpret_cast<const float4 *>(src.f[0]);
    const float4 *f4 = reinterpret_cast<const float4 *>(src.f[1]);
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < P.C / 4u; q += stride) {
      const float4 a = __ldg(o4 + q), b = __ldg(f4 + q);
      reinterpret_cast<float4 *>(B.zO)[q] = a;
      reinterpret_cast<float4 *>(B.zF)[q] = b;
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        bad |= !(av[j] >= 0.0f && av[j] <= 1.0f && bv[j] >= 0.0f && bv[j] <= 1.0f && av[j] + bv[j] <= 1.000001f);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&B.ctl->err, ERR_INPUT);
    return;
  }
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < P.C; c += stride) {
    const float a = __ldg(src.f[0] + c), b = __ldg(src.f[1] + c);
    B.zO[c] = a;
    B.zF[c] = b;
    if (kind == GRID_BERNOULLI) {  // z in {0, 1}; p_TP, p_FP in (0, 1); p_A in [0, 1]; p_c > 0
      const float pa = __ldg(src.f[2] + c), pfp = __ldg(src.f[3] + c), pc = __ldg(src.f[4] + c);
      B.pA[c] = pa;
      B.zv[c] = pfp;
      B.sgv[c] = pc;
      bad |= !(a == 0.0f || a == 1.0f);
      bad |= !(b > 0.0f && b < 1.0f && pfp > 0.0f && pfp < 1.0f);
      bad |= !(pa >= 0.0f && pa <= 1.0f);
      bad |= !(pc > 0.0f && pc < 3.0e38f);
      continue;
    }
    bad |= !(a >= 0.0f && a <= 1.0f && b >= 0.0f && b <= 1.0f && a + b <= 1.000001f);
    if (kind == GRID_RADAR) {
      const float pa = __ldg(src.f[2] + c), zv = __ldg(src.f[3] + c), sg = __ldg(src.f[4] + c);
      B.pA[c] = pa;
      B.zv[c] = zv;
      B.sgv[c] = sg;
      bad |= !(pa >= 0.0f && pa <= 1.0f);
      bad |= (pa > 0.0f) && !(sg > 0.0f);
      bad |= !(fabsf(zv) < 3.0e38f);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&B.ctl->err, ERR_INPUT);
}

// ====================================================================================
// Ego-motion compensation (filters created with DOG_EGO).  The grid moves with the
// vehicle: between two frames the vehicle moved by d = (dx, dy) in the previous grid's
// axes and turned by theta about the sensor position q.  A posterior particle enters the
// new grid at p' = q + R(-theta) (p - q - d) with velocity v' = R(-theta) v (k_predict,
// before the process model); the free mass carried over is read, for each new cell, at the
// old cell under its centre q + R(theta) (c - q) + d (k_ego_warp; 0 outside the old grid).
// ====================================================================================
constexpr uint32_t FLAG_EGO = 0x20u, FLAG_FULL = 0x40u;

__global__ void k_set_ego(DevCtl *ctl, uint32_t on, float c, float s, float dx, float dy) {
  ctl->ego_on = on;
  ctl->ego_c = c;
  ctl->ego_s = s;
  ctl->ego_dx = dx;
  ctl->ego_dy = dy;
}

struct Ego {
  float c, s, dx, dy;
};

__device__ __forceinline__ void ego_transform(const KParams &P, const Ego &E, float4 &st) {
  const float rx = __fsub_rn(__fsub_rn(st.x, P.sensor_x), E.dx);
  const float ry = __fsub_rn(__fsub_rn(st.y, P.sensor_y), E.dy);
  st.x = __fadd_rn(P.sensor_x, __fadd_rn(__fmul_rn(E.c, rx), __fmul_rn(E.s, ry)));
  st.y = __fadd_rn(P.sensor_y, __fsub_rn(__fmul_rn(E.c, ry), __fmul_rn(E.s, rx)));
  const float vx = st.z, vy = st.w;
  st.z = __fadd_rn(__fmul_rn(E.c, vx), __fmul_rn(E.s, vy));
  st.w = __fsub_rn(__fmul_rn(E.c, vy), __fmul_rn(E.s, vx));
}

__device__ __forceinline__ void ego_warp_body(const KParams &P, const DevBufs &B, uint32_t blk, uint32_t nblk) {
  const DevCtl *ctl = B.ctl;
  const bool on = ctl->ego_on != 0u;
  const Ego E{ctl->ego_c, ctl->ego_s, ctl->ego_dx, ctl->ego_dy};
  const uint32_t stride = nblk * blockDim.x;
  const float Wf = (float)P.W, Hf = (float)P.H;
  for (uint32_t c = blk * blockDim.x + threadIdx.x; c < P.C; c += stride) {
    float v;
    if (!on) {
      v = B.mF[c];
    } else {
      const uint32_t row = c / (uint32_t)P.W, col = c - row * (uint32_t)P.W;
      const float ux = __fsub_rn(__fmul_rn(__fadd_rn((float)col, 0.5f), P.s), P.sensor_x);
      const float uy = __fsub_rn(__fmul_rn(__fadd_rn((float)row, 0.5f), P.s), P.sensor_y);
      const float ox = __fadd_rn(__fadd_rn(P.sensor_x, __fsub_rn(__fmul_rn(E.c, ux), __fmul_rn(E.s, uy))), E.dx);
      const float oy = __fadd_rn(__fadd_rn(P.sensor_y, __fadd_rn(__fmul_rn(E.s, ux), __fmul_rn(E.c, uy))), E.dy);
      const float fx = __fdiv_rn(ox, P.s), fy = __fdiv_rn(oy, P.s);
      const bool in = fx >= 0.0f && fx < Wf && fy >= 0.0f && fy < Hf;
      v = in ? B.mF[(uint32_t)(int)fy * (uint32_t)P.W + (uint32_t)(int)fx] : 0.0f;
    }
    B.mF_warp[c] = v;
  }
}
__global__ void k_ego_warp(KParams P, DevBufs B) { ego_warp_body(P, B, blockIdx.x, gridDim.x); }

// ====================================================================================
// k_predict (Alg. 1): Eq. process with per-frame Gaussian noise, Eq. particle_persistence,
// cell index floor(x/s), floor(y/s) (outside the grid: nearest border cell, weight 0).
// Each block handles 4096 particles, 4 per thread per round with 16-byte accesses, and
// accumulates the digit histograms of all sort passes in shared memory.
// ====================================================================================
constexpr int PRED_BLOCK = 256, PRED_ROUNDS = 4, PRED_TILE = PRED_BLOCK * 4 * PRED_ROUNDS;

// key gets bit 31 set when the particle left the grid (its weight is then 0); the sort
// moves that bit from the cell index to the particle index (see k_sort_pass)
constexpr uint32_t OUT_OF_GRID = 0x80000000u;

__device__ __forceinline__ void predict_one(const KParams &P, const PhiloxKeys &PK, uint32_t i, uint32_t frame,
                                            float T, float4 &st, float &w, uint32_t &key) {
  float &x = st.x, &y = st.y, &vx = st.z, &vy = st.w;
  const U4 r = philox(i, frame, TAG_PREDICT, PK);
  float n0, n1, n2, n3;
  gauss2(r.a, r.b, n0, n1);
  gauss2(r.c, r.d, n2, n3);
  x = __fadd_rn(__fadd_rn(x, __fmul_rn(T, vx)), __fmul_rn(P.sigma_pos, n0));
  y = __fadd_rn(__fadd_rn(y, __fmul_rn(T, vy)), __fmul_rn(P.sigma_pos, n1));
  vx = __fadd_rn(vx, __fmul_rn(P.sigma_vel, n2));
  vy = __fadd_rn(vy, __fmul_rn(P.sigma_vel, n3));
  w = __fmul_rn(P.p_S, w);
  const float fx = __fdiv_rn(x, P.s), fy = __fdiv_rn(y, P.s);
  const float Wf = (float)P.W, Hf = (float)P.H;
  const bool in = fx >= 0.0f && fx < Wf && fy >= 0.0f && fy < Hf;
  const int col = !(fx >= 0.0f) ? 0 : (!(fx < Wf) ? P.W - 1 : (int)fx);
  const int row = !(fy >= 0.0f) ? 0 : (!(fy < Hf) ? P.H - 1 : (int)fy);
  if (!in) w = 0.0f;
  key = (uint32_t)row * (uint32_t)P.W + (uint32_t)col;
  if (!in) key |= OUT_OF_GRID;
}

__device__ __forceinline__ void predict_body(const KParams &P, const DevBufs &B, uint32_t blk) {
  extern __shared__ uint32_t sh_hist[];  // [passes][radix]
  const uint32_t nh = (uint32_t)P.passes * P.radix;
  for (uint32_t k = threadIdx.x; k < nh; k += PRED_BLOCK) sh_hist[k] = 0u;
  __syncthreads();
  const uint32_t frame = this_frame(B.ctl);
  const float T = B.ctl->dt;
  const uint32_t mode = B.ctl->post_mode;
  const float w_res = B.ctl->w_new;
  const uint32_t mask = P.radix - 1u;
  const bool ego = (P.flags & FLAG_EGO) != 0u && B.ctl->ego_on != 0u;
  const Ego E{B.ctl->ego_c, B.ctl->ego_s, B.ctl->ego_dx, B.ctl->ego_dy};
  const PhiloxKeys PK = philox_keys(P.seed_lo, P.seed_hi);
  for (int rnd = 0; rnd < PRED_ROUNDS; ++rnd) {
    const uint32_t i0 = blk * PRED_TILE + (uint32_t)rnd * (PRED_BLOCK * 4) + threadIdx.x * 4;
    uint32_t key[4];
    bool valid[4];
    if (i0 + 4 <= P.nu) {
      float4 s0, s1, s2, s3, w;
      if (mode == POST_DIRECT) {
        s0 = B.Os[i0]; s1 = B.Os[i0 + 1]; s2 = B.Os[i0 + 2]; s3 = B.Os[i0 + 3];
        w = *reinterpret_cast<const float4 *>(B.Bw + i0);
      } else {  // the records of the four particles' sources; equal weights
        const uint4 j = *reinterpret_cast<const uint4 *>(B.Bsrc + i0);
        s0 = j.x < P.nu ? B.Os[j.x] : B.bs[j.x - P.nu];
        s1 = j.y < P.nu ? B.Os[j.y] : B.bs[j.y - P.nu];
        s2 = j.z < P.nu ? B.Os[j.z] : B.bs[j.z - P.nu];
        s3 = j.w < P.nu ? B.Os[j.w] : B.bs[j.w - P.nu];
        w = make_float4(w_res, w_res, w_res, w_res);
      }
      if (ego) {  // into the new frame's grid first
        ego_transform(P, E, s0);
        ego_transform(P, E, s1);
        ego_transform(P, E, s2);
        ego_transform(P, E, s3);
      }
      predict_one(P, PK, i0 + 0, frame, T, s0, w.x, key[0]);
      predict_one(P, PK, i0 + 1, frame, T, s1, w.y, key[1]);
      predict_one(P, PK, i0 + 2, frame, T, s2, w.z, key[2]);
      predict_one(P, PK, i0 + 3, frame, T, s3, w.w, key[3]);
      B.As[i0] = s0;
      B.As[i0 + 1] = s1;
      B.As[i0 + 2] = s2;
      B.As[i0 + 3] = s3;
      *reinterpret_cast<float4 *>(B.Aw + i0) = w;
      *reinterpret_cast<uint4 *>(B.key_pred + i0) = make_uint4(key[0], key[1], key[2], key[3]);
      valid[0] = valid[1] = valid[2] = valid[3] = true;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t i = i0 + k;
        valid[k] = i < P.nu;
        key[k] = 0u;
        if (valid[k]) {
          float4 s = posterior_record(P, B, mode, i);
          if (ego) ego_transform(P, E, s);
          float w = mode == POST_DIRECT ? B.Bw[i] : w_res;
          predict_one(P, PK, i, frame, T, s, w, key[k]);
          B.As[i] = s;
          B.Aw[i] = w;
          B.key_pred[i] = key[k];
        }
      }
    }
    // digit histograms: the thread's four consecutive particles mostly share a cell (the
    // posterior is in cell order), so runs of equal digits are added with one atomic each
    for (int p = 0; p < P.passes; ++p) {
      uint32_t cur = 0xffffffffu, cnt = 0u;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!valid[k]) continue;
        const uint32_t d = (key[k] >> (p * P.dbits)) & mask;
        if (d != cur) {
          if (cnt) atomicAdd(&sh_hist[p * P.radix + cur], cnt);
          cur = d;
          cnt = 0u;
        }
        ++cnt;
      }
      if (cnt) atomicAdd(&sh_hist[p * P.radix + cur], cnt);
    }
  }
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < nh; k += PRED_BLOCK) {
    const uint32_t v = sh_hist[k];
    if (v) atomicAdd(&B.hist[(k / P.radix) * 2048u + (k % P.radix)], v);
  }
  // this block's keys are tile blk of the first sort pass: its first-pass digit counts
  for (uint32_t d = threadIdx.x; d < P.radix; d += PRED_BLOCK)
    B.dcnt[(size_t)d * P.tiles_sort + blk] = sh_hist[d];
}
__global__ void __launch_bounds__(PRED_BLOCK) k_predict(KParams P, DevBufs B) { predict_body(P, B, blockIdx.x); }

// ====================================================================================
// Sort (Alg. 2): LSD radix sort of (cell index, particle index) pairs on digits of up to 11
// bits, reduce-then-scan: every pass works on fixed tiles of 4096 pairs, and the output
// offset of each (digit, tile) is known before the pass starts, so no block waits for
// another.
//   - digit counts per tile, stored digit-major ([pass][digit][tile]): k_predict writes the
//     first pass's (its blocks are that pass's tiles); k_sort_count counts a later pass's
//     tiles in the output of the pass before;
//   - k_sort_offsets turns one pass's counts into global offsets, in place: start of the
//     digit (prefix of the digit histogram) + the digit's count in all earlier tiles;
//   - k_sort_pass ranks its tile stably in shared memory (warp-private digit counters with
//     match.any) and writes each digit's run contiguously at its offset.
// ====================================================================================
constexpr int SORT_BLOCK = 512, SORT_ITEMS = 8, SORT_WARPS = SORT_BLOCK / 32,
              SORT_TILE = SORT_BLOCK * SORT_ITEMS;
static_assert(PRED_TILE == SORT_TILE, "k_predict's blocks are the first sort pass's tiles");

__host__ __device__ constexpr size_t sort_smem_bytes(uint32_t radix) {
  // ranking: per-warp u16 histograms, later reused for the staged keys and values
  return ((size_t)SORT_WARPS * radix * 2 > (size_t)SORT_TILE * 8 ? (size_t)SORT_WARPS * radix * 2
                                                                  : (size_t)SORT_TILE * 8) +
         (size_t)3 * radix * 4 + 128;
}

// exclusive scan of n <= 2048 values in shared memory by SORT_BLOCK threads
__device__ void block_excl_scan_u32(const uint32_t *in, uint32_t *out, uint32_t n, uint32_t *s_warp) {
  const uint32_t per = (n + SORT_BLOCK - 1) / SORT_BLOCK;  // <= 4
  const uint32_t b = threadIdx.x * per;
  uint32_t loc = 0;
  for (uint32_t k = 0; k < per; ++k)
    if (b + k < n) loc += in[b + k];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, inc, o);
    if (lane >= (uint32_t)o) inc += t;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the SORT_WARPS warp totals
    const uint32_t v = lane < (uint32_t)SORT_WARPS ? s_warp[lane] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < SORT_WARPS; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, x, o);
      if (lane >= (uint32_t)o) x += t;
    }
    __syncwarp();
    if (lane < (uint32_t)SORT_WARPS) s_warp[lane] = x - v;
  }
  __syncthreads();
  uint32_t run = s_warp[warp] + inc - loc;
  for (uint32_t k = 0; k < per; ++k)
    if (b + k < n) {
      const uint32_t v = in[b + k];
      out[b + k] = run;
      run += v;
    }
  __syncthreads();
}

// k_sort_count: digit counts of one pass's tiles in the output of the pass before.  A block
// counts ct consecutive tiles (ct = 1, 2, 4 or 8, the most that still leaves two blocks per
// SM; 16-byte key loads, shared-memory counters per tile), so that each digit's counts of
// those tiles are contiguous in its row of the digit-major table and go out as 16-byte
// (or 8-byte) stores instead of ct separate 4-byte ones
constexpr int COUNT_BLOCK = 512, COUNT_TILES = 8;  // at most

__host__ __device__ constexpr size_t count_smem_bytes(uint32_t radix, uint32_t ct) {
  return (size_t)ct * radix * 4;
}
inline uint32_t count_tiles_per_block(uint32_t tiles, int sms) {
  uint32_t ct = COUNT_TILES;
  while (ct > 1u && tiles / ct < 2u * (uint32_t)sms) ct >>= 1;
  return ct;
}

__device__ __forceinline__ void sort_count_body(const KParams &P, const DevBufs &B, const uint32_t *__restrict__ keys,
                                                int pass, uint32_t ct, uint32_t blk) {
  extern __shared__ uint32_t sh_cnt[];  // [ct][radix]
  const uint32_t radix = P.radix, mask = radix - 1u;
  const int shift = pass * P.dbits;
  for (uint32_t k = threadIdx.x; k < ct * radix; k += COUNT_BLOCK) sh_cnt[k] = 0u;
  __syncthreads();
  const uint32_t t0 = blk * ct;
  const uint32_t base = t0 * SORT_TILE;
  const uint32_t end = min(base + ct * SORT_TILE, P.nu);
  // four consecutive keys per thread and access (the same tile: SORT_TILE % 4 == 0), four
  // such accesses loaded before any is counted; equal neighbouring digits are added together
  constexpr int G = 4;
  for (uint32_t i0 = base + 4 * threadIdx.x; i0 < end; i0 += G * 4 * COUNT_BLOCK) {
    uint32_t k4[G][4];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const uint32_t i = i0 + g * 4 * COUNT_BLOCK;
      if (i + 4 <= end) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(keys + i));
        k4[g][0] = v.x; k4[g][1] = v.y; k4[g][2] = v.z; k4[g][3] = v.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) k4[g][j] = i + j < end ? __ldg(keys + i + j) : 0xffffffffu;
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const uint32_t i = i0 + g * 4 * COUNT_BLOCK;
      if (i >= end) break;
      uint32_t *cnt = sh_cnt + ((i - base) / SORT_TILE) * radix;
      uint32_t cur = 0xffffffffu, run = 0u;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (k4[g][j] == 0xffffffffu) continue;  // past the end
        const uint32_t d = (k4[g][j] >> shift) & mask;
        if (d != cur) {
          if (run) atomicAdd(cnt + cur, run);
          cur = d;
          run = 0u;
        }
        ++run;
      }
      if (run) atomicAdd(cnt + cur, run);
    }
  }
  __syncthreads();
  uint32_t *col = B.dcnt + (size_t)pass * radix * P.tiles_sort;
  const uint32_t nt = min(ct, P.tiles_sort - t0);
  // rows start on 16-byte (8-byte) boundaries when tiles_sort is a multiple of 4 (2), and so
  // does this block's run t0 = blk * ct
  const bool v4 = nt == ct && ct % 4u == 0u && P.tiles_sort % 4u == 0u;
  const bool v2 = nt == ct && ct == 2u && P.tiles_sort % 2u == 0u;
  for (uint32_t d = threadIdx.x; d < radix; d += COUNT_BLOCK) {
    uint32_t *row = col + (size_t)d * P.tiles_sort + t0;
    if (v4) {
      for (uint32_t t = 0; t < ct; t += 4)
        *reinterpret_cast<uint4 *>(row + t) = make_uint4(sh_cnt[t * radix + d], sh_cnt[(t + 1) * radix + d],
                                                         sh_cnt[(t + 2) * radix + d], sh_cnt[(t + 3) * radix + d]);
    } else if (v2) {
      *reinterpret_cast<uint2 *>(row) = make_uint2(sh_cnt[d], sh_cnt[radix + d]);
    } else {
      for (uint32_t t = 0; t < nt; ++t) row[t] = sh_cnt[t * radix + d];
    }
  }
}
__global__ void __launch_bounds__(COUNT_BLOCK) k_sort_count(KParams P, DevBufs B,
                                                            const uint32_t *__restrict__ keys, int pass,
                                                            uint32_t ct) {
  sort_count_body(P, B, keys, pass, ct, blockIdx.x);
}

// k_sort_offsets: for one pass, counts[d][t] -> (sum of the histogram below digit d) +
// sum_{t' < t} counts[d][t'], in place.  One block per digit; thread k owns a contiguous run
// of tiles, held in registers (read once, 16-byte loads where the row allows), and the
// block scans the runs' totals.  OFF_PER, the most tiles a thread holds, is the smallest of
// 4, 8 and 16 that covers the filter's tiles (fewer registers: more blocks per SM).
constexpr int OFF_BLOCK = 256, OFF_WARPS = OFF_BLOCK / 32;

// the register run length for T sort tiles (T > 16 OFF_BLOCK takes the run from memory)
inline int offsets_per(uint32_t T) {
  const uint32_t per = (T + OFF_BLOCK - 1) / OFF_BLOCK;
  return per <= 4u ? 4 : (per <= 8u ? 8 : 16);
}

template <int OFF_PER>
__device__ __forceinline__ void sort_offsets_body(const KParams &P, const DevBufs &B, int pass, uint32_t blk) {
  __shared__ uint32_t s_h[OFF_WARPS], s_t[OFF_WARPS];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t d = blk;
  const uint32_t T = P.tiles_sort;
  const uint32_t *hist = B.hist + pass * 2048u;
  uint32_t *M = B.dcnt + ((size_t)pass * P.radix + d) * T;
  const uint32_t per = (T + OFF_BLOCK - 1) / OFF_BLOCK;  // tiles per thread
  const uint32_t t0 = threadIdx.x * per;
  // this thread's share of the histogram below d
  uint32_t hsum = 0;
  for (uint32_t e = threadIdx.x; e < d; e += OFF_BLOCK) hsum += __ldg(hist + e);
  // rows of up to OFF_PER tiles per thread stay in registers; the 16-byte path needs the
  // row and the thread's run to start on 16-byte boundaries
  const bool in_regs = per <= (uint32_t)OFF_PER;
  const bool vec = in_regs && (per % 4u) == 0u && (T % 4u) == 0u;
  uint32_t c[OFF_PER];
  uint32_t tsum = 0;
  if (vec) {
#pragma unroll
    for (int j = 0; j < OFF_PER; j += 4) {
      const uint32_t t = t0 + j;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if ((uint32_t)j < per && t < T) v = *reinterpret_cast<const uint4 *>(M + t);  // T % 4 == 0
      c[j] = v.x; c[j + 1] = v.y; c[j + 2] = v.z; c[j + 3] = v.w;
    }
  } else if (in_regs) {
#pragma unroll
    for (int j = 0; j < OFF_PER; ++j) {
      const uint32_t t = t0 + j;
      c[j] = ((uint32_t)j < per && t < T) ? M[t] : 0u;
    }
  } else {
    for (uint32_t j = 0; j < per; ++j) {
      const uint32_t t = t0 + j;
      tsum += t < T ? M[t] : 0u;
    }
  }
  if (in_regs) {
#pragma unroll
    for (int j = 0; j < OFF_PER; ++j) tsum += c[j];
  }
  // block: total of hsum, exclusive prefix of tsum
  uint32_t tinc = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    hsum += __shfl_xor_sync(FULL, hsum, o);
    const uint32_t y = __shfl_up_sync(FULL, tinc, o);
    if (lane >= (uint32_t)o) tinc += y;
  }
  if (lane == 31) {
    s_h[warp] = hsum;
    s_t[warp] = tinc;
  }
  __syncthreads();
  uint32_t run = tinc - tsum;
  for (uint32_t w = 0; w < OFF_WARPS; ++w) {
    run += s_h[w];
    if (w < warp) run += s_t[w];
  }
  if (vec) {
#pragma unroll
    for (int j = 0; j < OFF_PER; j += 4) {
      const uint32_t t = t0 + j;
      uint4 v;
      v.x = run; run += c[j];
      v.y = run; run += c[j + 1];
      v.z = run; run += c[j + 2];
      v.w = run; run += c[j + 3];
      if ((uint32_t)j < per && t < T) *reinterpret_cast<uint4 *>(M + t) = v;
    }
  } else if (in_regs) {
#pragma unroll
    for (int j = 0; j < OFF_PER; ++j) {
      const uint32_t t = t0 + j;
      if ((uint32_t)j < per && t < T) M[t] = run;
      run += c[j];
    }
  } else {
    for (uint32_t j = 0; j < per; ++j) {
      const uint32_t t = t0 + j;
      if (t >= T) break;
      const uint32_t v = M[t];
      M[t] = run;
      run += v;
    }
  }
}
template <int OFF_PER>
__global__ void __launch_bounds__(OFF_BLOCK, OFF_PER <= 4 ? 8 : 1) k_sort_offsets(KParams P, DevBufs B, int pass) {
  sort_offsets_body<OFF_PER>(P, B, pass, blockIdx.x);
}

__device__ __forceinline__ void sort_pass_body(const KParams &P, const DevBufs &B, const uint32_t *__restrict__ keys_in,
                                               const uint32_t *__restrict__ vals_in, uint32_t *__restrict__ keys_out,
                                               uint32_t *__restrict__ vals_out, int pass, uint32_t blk) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t radix = P.radix;
  const size_t big = sort_smem_bytes(radix) - (size_t)3 * radix * 4 - 128;
  uint16_t *s_whist = reinterpret_cast<uint16_t *>(smem);      // [warps][radix]
  uint2 *s_kv = reinterpret_cast<uint2 *>(smem);               // [tile] (key, value), after ranking
  uint32_t *s_cnt = reinterpret_cast<uint32_t *>(smem + big);  // [radix]
  uint32_t *s_excl = s_cnt + radix;
  uint32_t *s_base = s_excl + radix;
  uint32_t *s_misc = s_base + radix;  // [32]: warp sums

  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile = blk;
  const int shift = pass * P.dbits;
  const uint32_t mask = radix - 1u;
  // global output offset of this tile's digits (radix <= 2048)
  constexpr int DPT = (2048 + SORT_BLOCK - 1) / SORT_BLOCK;  // digits per thread, at most
  const uint32_t *off = B.dcnt + (size_t)pass * radix * P.tiles_sort + tile;
  uint32_t offr[DPT];
#pragma unroll
  for (int j = 0; j < DPT; ++j) {
    const uint32_t d = tid + j * SORT_BLOCK;
    offr[j] = d < radix ? __ldg(off + (size_t)d * P.tiles_sort) : 0u;
  }
  // the pass's digit histogram was read by k_sort_offsets: cleared here for the next
  // frame's prediction, which adds into it
  if (tile == 0u)
    for (uint32_t d = tid; d < radix; d += SORT_BLOCK) B.hist[pass * 2048u + d] = 0u;
  // warp counters cleared with 16-byte stores (SORT_WARPS * radix * 2 bytes, a multiple of 16)
  for (uint32_t k = tid; k < SORT_WARPS * radix / 8; k += SORT_BLOCK)
    reinterpret_cast<uint4 *>(s_whist)[k] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();

  // load: warp w covers positions [w*256, w*256+256) of the tile, item k at k*32 + lane
  uint32_t key[SORT_ITEMS], val[SORT_ITEMS];
  const uint32_t base = tile * SORT_TILE + warp * (32 * SORT_ITEMS);
  if (vals_in) {  // block-uniform
#pragma unroll
    for (int k = 0; k < SORT_ITEMS; ++k) {
      const uint32_t pos = base + k * 32 + lane;
      const bool ok = pos < P.nu;
      key[k] = ok ? __ldg(keys_in + pos) : 0xffffffffu;
      val[k] = ok ? __ldg(vals_in + pos) : 0u;
    }
  } else {  // first pass: the out-of-grid bit moves from the cell index to the particle index
#pragma unroll
    for (int k = 0; k < SORT_ITEMS; ++k) {
      const uint32_t pos = base + k * 32 + lane;
      const bool ok = pos < P.nu;
      const uint32_t raw = ok ? __ldg(keys_in + pos) : 0xffffffffu;
      key[k] = ok ? (raw & ~OUT_OF_GRID) : 0xffffffffu;
      val[k] = ok ? (pos | (raw & OUT_OF_GRID)) : 0u;
    }
  }
  // stable rank within the warp, item by item
  uint32_t rk[SORT_ITEMS];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int k = 0; k < SORT_ITEMS; ++k) {
    const uint32_t d = (key[k] >> shift) & mask;
    const uint32_t peers = __match_any_sync(FULL, d);
    const uint16_t pre = s_whist[warp * radix + d];
    __syncwarp();
    if ((peers & lt) == 0u) s_whist[warp * radix + d] = (uint16_t)(pre + __popc(peers));
    __syncwarp();
    rk[k] = pre + __popc(peers & lt);
  }
  __syncthreads();
  // per digit: exclusive offsets of the warps and the tile's count.  Two neighbouring
  // digits' u16 counters are scanned together as one u32 (a digit's count in a tile is at
  // most 4096, so the low half never carries into the high one)
  {
    const uint32_t *wh = reinterpret_cast<const uint32_t *>(s_whist);
    uint32_t *wh_out = reinterpret_cast<uint32_t *>(s_whist);
    const uint32_t half = radix >> 1;  // digit pairs per warp row (radix >= 2)
    for (uint32_t pr = tid; pr < half; pr += SORT_BLOCK) {
      uint32_t run = 0;
#pragma unroll 4
      for (int w = 0; w < SORT_WARPS; ++w) {
        const uint32_t c = wh[w * half + pr];
        wh_out[w * half + pr] = run;
        run += c;
      }
      s_cnt[2 * pr] = run & 0xffffu;
      s_cnt[2 * pr + 1] = run >> 16;
    }
  }
#pragma unroll
  for (int j = 0; j < DPT; ++j) {
    const uint32_t d = tid + j * SORT_BLOCK;
    if (d < radix) s_base[d] = offr[j];
  }
  __syncthreads();
  block_excl_scan_u32(s_cnt, s_excl, radix, s_misc);
  // tile-local sorted position of each key
  uint32_t lpos[SORT_ITEMS];
#pragma unroll
  for (int k = 0; k < SORT_ITEMS; ++k) {
    const uint32_t d = (key[k] >> shift) & mask;
    lpos[k] = s_excl[d] + s_whist[warp * radix + d] + rk[k];
  }
  for (uint32_t d = tid; d < radix; d += SORT_BLOCK) s_base[d] -= s_excl[d];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < SORT_ITEMS; ++k) s_kv[lpos[k]] = make_uint2(key[k], val[k]);
  __syncthreads();
  // scatter: runs of equal digits are contiguous in shared memory and in the output
  for (uint32_t p = tid; p < SORT_TILE; p += SORT_BLOCK) {
    const uint2 kv = s_kv[p];
    const uint32_t gp = s_base[(kv.x >> shift) & mask] + p;
    if (gp < P.nu) {
      keys_out[gp] = kv.x;
      vals_out[gp] = kv.y;
    }
  }
}
__global__ void __launch_bounds__(SORT_BLOCK, 2)
    k_sort_pass(KParams P, DevBufs B, const uint32_t *__restrict__ keys_in,
                const uint32_t *__restrict__ vals_in, uint32_t *__restrict__ keys_out,
                uint32_t *__restrict__ vals_out, int pass) {
  sort_pass_body(P, B, keys_in, vals_in, keys_out, vals_out, pass, blockIdx.x);
}

// ====================================================================================
// Segmented sums over the sorted particles.  A thread owns ITEMS consecutive sorted
// positions; segments are the cells (runs of equal keys).  A block reduces its tile with a
// block-wide segmented scan.  A segment inside one tile is finished by the thread holding
// its last particle; a segment that crosses tile boundaries leaves one piece per tile,
// added with 64-bit integer atomics (exact, so their order does not matter) to a per-cell
// accumulator that is read and cleared after all pieces are in.  k_segsum also writes
// the predicted particles in sorted order, so later kernels stream them contiguously.  No block waits for
// another block.
// ====================================================================================
// 1024-position tiles: smaller tiles keep more blocks (and their gathers) in flight on
// each SM than 2048-position ones, at the price of more cells crossing a tile edge
constexpr int SEG_BLOCK = 256, SEG_ITEMS = 4, SEG_TILE = SEG_BLOCK * SEG_ITEMS;

// shared-memory index padded by one element per SEG_ITEMS: a thread's blocked run starts
// SEG_ITEMS + 1 elements after its neighbour's (odd, so a warp hits 32 distinct banks)
__device__ __forceinline__ uint32_t seg_pad(uint32_t m) { return m + m / SEG_ITEMS; }
constexpr int SEG_PADDED = SEG_TILE + SEG_TILE / SEG_ITEMS;

template <int N, typename V = unsigned long long>
struct Seg {
  uint32_t f;  // a segment head lies in the covered range
  V v[N];
};

// (a then b): a head in b cuts off a
template <int N, typename V>
__device__ __forceinline__ Seg<N, V> seg_combine(const Seg<N, V> &a, const Seg<N, V> &b) {
  Seg<N, V> r;
  r.f = a.f | b.f;
#pragma unroll
  for (int k = 0; k < N; ++k) r.v[k] = b.f ? b.v[k] : a.v[k] + b.v[k];
  return r;
}

template <int N, typename V>
__device__ __forceinline__ Seg<N, V> seg_shfl_up(const Seg<N, V> &a, int o) {
  Seg<N, V> r;
  r.f = __shfl_up_sync(FULL, a.f, o);
#pragma unroll
  for (int k = 0; k < N; ++k) r.v[k] = __shfl_up_sync(FULL, a.v[k], o);
  return r;
}

template <int N, typename V>
__device__ __forceinline__ Seg<N, V> seg_zero(const Seg<N, V> &) {
  Seg<N, V> r;
  r.f = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) r.v[k] = V(0);
  return r;
}

// five compensated (double-float) moment sums under one head flag, and the same with the
// fixed-point weight sum of the segment pass
struct SegMom {
  uint32_t f;
  DF m[5];
};
struct SegQM {
  uint32_t f;
  unsigned long long q;
  DF m[5];
};
__device__ __forceinline__ SegMom seg_combine(const SegMom &a, const SegMom &b) {
  SegMom r;
  r.f = a.f | b.f;
#pragma unroll
  for (int k = 0; k < 5; ++k) r.m[k] = b.f ? b.m[k] : df_add(a.m[k], b.m[k]);
  return r;
}
__device__ __forceinline__ SegQM seg_combine(const SegQM &a, const SegQM &b) {
  SegQM r;
  r.f = a.f | b.f;
  r.q = b.f ? b.q : a.q + b.q;
#pragma unroll
  for (int k = 0; k < 5; ++k) r.m[k] = b.f ? b.m[k] : df_add(a.m[k], b.m[k]);
  return r;
}
template <typename S>
__device__ __forceinline__ void shfl_moments(S &r, const S &a, int o) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    r.m[k].hi = __shfl_up_sync(FULL, a.m[k].hi, o);
    r.m[k].lo = __shfl_up_sync(FULL, a.m[k].lo, o);
  }
}
__device__ __forceinline__ SegMom seg_shfl_up(const SegMom &a, int o) {
  SegMom r;
  r.f = __shfl_up_sync(FULL, a.f, o);
  shfl_moments(r, a, o);
  return r;
}
__device__ __forceinline__ SegQM seg_shfl_up(const SegQM &a, int o) {
  SegQM r;
  r.f = __shfl_up_sync(FULL, a.f, o);
  r.q = __shfl_up_sync(FULL, a.q, o);
  shfl_moments(r, a, o);
  return r;
}
__device__ __forceinline__ SegMom seg_zero(const SegMom &) {
  SegMom r;
  r.f = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k) r.m[k] = DF{0.0f, 0.0f};
  return r;
}
__device__ __forceinline__ SegQM seg_zero(const SegQM &) {
  SegQM r;
  r.f = 0;
  r.q = 0ull;
#pragma unroll
  for (int k = 0; k < 5; ++k) r.m[k] = DF{0.0f, 0.0f};
  return r;
}

// Block-wide exclusive segmented scan of per-thread aggregates (SEG_BLOCK threads).
template <typename S>
__device__ S block_seg_excl(const S &x, S *s_w /* [SEG_BLOCK/32 + 1] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  S inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const S t = seg_shfl_up(inc, o);
    if (lane >= o) inc = seg_combine(t, inc);
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    S run = seg_zero(x);
    for (int w = 0; w < SEG_BLOCK / 32; ++w) {
      const S t = s_w[w];
      s_w[w] = run;
      run = seg_combine(run, t);
    }
  }
  __syncthreads();
  S prev = seg_shfl_up(inc, 1);
  if (lane == 0) prev = seg_zero(x);
  return seg_combine(s_w[warp], prev);
}

// radial-velocity likelihood g (constant factor dropped; it cancels in mu_A)
__device__ __forceinline__ float radar_lik(const KParams &P, float x, float y, float vx, float vy,
                                           float zv, float sg) {
  const float dx = __fsub_rn(x, P.sensor_x), dy = __fsub_rn(y, P.sensor_y);
  const float r = __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
  float vr = 0.0f;
  if (r > 0.0f) vr = __fdiv_rn(__fadd_rn(__fmul_rn(dx, vx), __fmul_rn(dy, vy)), r);
  const float d = __fdiv_rn(__fsub_rn(vr, zv), sg);
  return exp_f(__fmul_rn(-0.5f, __fmul_rn(d, d)));
}

// load ITEMS consecutive u32 at position j0 (16-byte accesses when the run is interior)
template <int ITEMS>
__device__ __forceinline__ void load_run(const uint32_t *p, uint32_t j0, uint32_t n, uint32_t (&o)[ITEMS],
                                         uint32_t fill) {
  if (j0 + ITEMS <= n) {
#pragma unroll
    for (int k = 0; k < ITEMS; k += 4) {
      const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p + j0 + k));
      o[k] = v.x; o[k + 1] = v.y; o[k + 2] = v.z; o[k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) o[k] = (j0 + k < n) ? __ldg(p + j0 + k) : fill;
  }
}

// ITEMS consecutive floats at position j0 (16-byte accesses when the run is interior)
template <int ITEMS>
__device__ __forceinline__ void load_runf(const float *p, uint32_t j0, uint32_t n, float (&o)[ITEMS]) {
  if (j0 + ITEMS <= n) {
#pragma unroll
    for (int k = 0; k < ITEMS; k += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(p + j0 + k));
      o[k] = v.x; o[k + 1] = v.y; o[k + 2] = v.z; o[k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) o[k] = (j0 + k < n) ? __ldg(p + j0 + k) : 0.0f;
  }
}
template <int ITEMS>
__device__ __forceinline__ void store_run(float *p, uint32_t j0, uint32_t n, const float (&v)[ITEMS]) {
  if (j0 + ITEMS <= n) {
#pragma unroll
    for (int k = 0; k < ITEMS; k += 4)
      *reinterpret_cast<float4 *>(p + j0 + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
      if (j0 + k < n) p[j0 + k] = v[k];
  }
}

// moment terms of one particle as exact double-float products: w v_x, w v_y, w v_x^2,
// w v_y^2, w v_x v_y (w v_x and w v_y exact; the second products carry the first's low part)
__device__ __forceinline__ void moment_terms(float w, float vx, float vy, DF (&m)[5]) {
  const DF mx = two_prod(w, vx), my = two_prod(w, vy);
  m[0] = mx;
  m[1] = my;
  const DF xx = two_prod(mx.hi, vx), yy = two_prod(my.hi, vy), xy = two_prod(mx.hi, vy);
  m[2] = DF{xx.hi, __fmaf_rn(mx.lo, vx, xx.lo)};
  m[3] = DF{yy.hi, __fmaf_rn(my.lo, vy, yy.lo)};
  m[4] = DF{xy.hi, __fmaf_rn(mx.lo, vy, xy.lo)};
}

// Eq. mean_x, var_x, covar_xy from the expectations E[vx], E[vy], E[vx^2], E[vy^2], E[vx vy]
// under the cell-normalised weights (double-float), each result rounded once to binary32;
// variances clamped at 0
__device__ __forceinline__ void moments_of_expectations(const DF (&E)[5], float (&o)[5]) {
  o[0] = df_to_f(E[0]);
  o[1] = df_to_f(E[1]);
  o[2] = fmaxf(df_to_f(df_sub(E[2], df_mul(E[0], E[0]))), 0.0f);
  o[3] = fmaxf(df_to_f(df_sub(E[3], df_mul(E[1], E[1]))), 0.0f);
  o[4] = df_to_f(df_sub(E[4], df_mul(E[0], E[1])));
}
// the moments from the sums of w v, ... over a cell, times the factor f / d (f >= 0, d > 0):
// E = sum (f / d), the factor once in double-float
__device__ __forceinline__ void moments_scaled(const DF (&m)[5], float f, float d, float (&o)[5]) {
  const DF k = df_div_f(DF{f, 0.0f}, d);
  DF E[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) E[i] = df_mul(m[i], k);
  moments_of_expectations(E, o);
}
__device__ __forceinline__ void moments_store(const DevBufs &B, uint32_t c, const float (&o)[5]) {
  B.mean_x[c] = o[0];
  B.mean_y[c] = o[1];
  B.var_x[c] = o[2];
  B.var_y[c] = o[3];
  B.cov[c] = o[4];
}

// a cell's head: S and the tag
__device__ __forceinline__ void csum_store_head(CellSum *r, unsigned long long S, uint32_t tag) {
  *reinterpret_cast<uint4 *>(r) = make_uint4((uint32_t)S, (uint32_t)(S >> 32), tag, 0u);
}
// the compensated moment sums of a cell finished in one tile
__device__ __forceinline__ void cmom_store(CellMom *r, const DF (&m)[5]) {
  float4 *q = reinterpret_cast<float4 *>(r);
  q[0] = make_float4(m[0].hi, m[1].hi, m[2].hi, m[3].hi);
  q[1] = make_float4(m[4].hi, m[0].lo, m[1].lo, m[2].lo);
  q[2] = make_float4(m[3].lo, m[4].lo, 0.0f, 0.0f);
}
__device__ __forceinline__ void cmom_load(const CellMom *r, DF (&m)[5]) {
  const float4 *q = reinterpret_cast<const float4 *>(r);
  const float4 a = q[0], b = q[1], c = q[2];
  m[0] = DF{a.x, b.y};
  m[1] = DF{a.y, b.z};
  m[2] = DF{a.z, b.w};
  m[3] = DF{a.w, c.x};
  m[4] = DF{b.x, c.y};
}

// k_segsum: cell ranges (Alg. 2) and S_c = sum of q40(w) (Eq. DS_particle_sum_pred as an
// exact fixed-point sum), plus A_c = sum of q40(g w) where the cell has a radar likelihood.
// tag[c] = 2 frame (finished here) or 2 frame + 1 (pieces in the accumulators).  The
// predicted state is gathered through the sort permutation into sorted order (Os, Ow) with
// consecutive lanes on consecutive sorted positions (neighbouring particles mostly come
// from neighbouring slots), and the fixed-point weights reach the blocked segmented scan
// through shared memory.  The radar filter also leaves each particle's likelihood g in wn
// (sorted order), where k_normalise reads it before it writes the normalised weight.
template <bool RADAR>
__device__ __forceinline__ void segsum_body(const KParams &P, const DevBufs &B, uint32_t blk) {
  constexpr int N = RADAR ? 2 : 1;
  __shared__ Seg<N> s_w[SEG_BLOCK / 32 + 1];
  __shared__ unsigned long long s_q[N][SEG_PADDED];
  const uint32_t tile = blk, frame = this_frame(B.ctl);
  const uint32_t base = tile * SEG_TILE;
  const uint32_t last_valid = min(base + SEG_TILE, P.nu) - 1u;
  // gather phase, warp-striped: position base + it*256 + threadIdx.x.  All permutation
  // loads are issued, then all record loads, then the stores, so that a thread keeps
  // SEG_ITEMS independent gathers in flight.
  // after a resampled frame every predicted weight is p_S w_new, or 0 for a particle that
  // left the grid (flagged in the particle index), so only the record is gathered
  const bool uniform = B.ctl->post_mode == POST_RESAMPLED;
  const float wu = __fmul_rn(P.p_S, B.ctl->w_new);
  const unsigned long long qwu = q40(wu);  // the fixed-point weight of every in-grid particle
  uint32_t gi[SEG_ITEMS];
#pragma unroll
  for (int it = 0; it < SEG_ITEMS; ++it) {
    const uint32_t j = base + it * SEG_BLOCK + threadIdx.x;
    gi[it] = j < P.nu ? __ldg(B.perm + j) : 0xffffffffu;
  }
  float4 st[SEG_ITEMS];
  float w[SEG_ITEMS];
#pragma unroll
  for (int it = 0; it < SEG_ITEMS; ++it) {
    st[it] = make_float4(0.f, 0.f, 0.f, 0.f);
    w[it] = 0.0f;
    if (gi[it] != 0xffffffffu) {
      const uint32_t i = gi[it] & ~OUT_OF_GRID;
      st[it] = __ldg(B.As + i);
      w[it] = uniform ? ((gi[it] & OUT_OF_GRID) ? 0.0f : wu) : __ldg(B.Aw + i);
    }
  }
#pragma unroll
  for (int it = 0; it < SEG_ITEMS; ++it) {
    const uint32_t m = it * SEG_BLOCK + threadIdx.x;
    const uint32_t j = base + m;
    unsigned long long q = 0ull, gq = 0ull;
    if (j < P.nu) {
      B.Os[j] = st[it];
      B.Ow[j] = w[it];
      q = uniform ? (w[it] > 0.0f ? qwu : 0ull) : q40(w[it]);
      if constexpr (RADAR) {
        const uint32_t c = __ldg(B.key_sorted + j);
        float g = 0.0f;
        if (__ldg(B.pA + c) > 0.0f) {
          g = radar_lik(P, st[it].x, st[it].y, st[it].z, st[it].w, __ldg(B.zv + c), __ldg(B.sgv + c));
          gq = q40(__fmul_rn(g, w[it]));
        }
        B.wn[j] = g;  // kept for k_normalise, which overwrites it with the normalised weight
      }
    }
    s_q[0][seg_pad(m)] = q;
    if constexpr (RADAR) s_q[N - 1][seg_pad(m)] = gq;
  }
  __syncthreads();
  // scan phase, blocked: a thread owns ITEMS consecutive positions
  const uint32_t j0 = base + threadIdx.x * SEG_ITEMS;
  uint32_t key[SEG_ITEMS];
  load_run<SEG_ITEMS>(B.key_sorted, j0, P.nu, key, 0xffffffffu);
  const uint32_t kprev = (j0 > 0 && j0 <= P.nu) ? __ldg(B.key_sorted + j0 - 1) : 0xfffffffeu;
  const uint32_t knext = (j0 + SEG_ITEMS < P.nu) ? __ldg(B.key_sorted + j0 + SEG_ITEMS) : 0xfffffffeu;
  unsigned long long v[SEG_ITEMS][N];
  uint32_t head = 0, tail = 0;
  Seg<N> agg;
  agg.f = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) agg.v[k] = 0ull;
#pragma unroll
  for (int it = 0; it < SEG_ITEMS; ++it) {
    const uint32_t j = j0 + it;
    const bool ok = j < P.nu;
    const uint32_t kp = it == 0 ? kprev : key[it - 1];
    const uint32_t kn = it == SEG_ITEMS - 1 ? knext : key[it + 1];
    const bool h = ok && (j == 0 || key[it] != kp);
    const bool t = ok && (j == P.nu - 1 || key[it] != kn);
    head |= (uint32_t)h << it;
    tail |= (uint32_t)t << it;
#pragma unroll
    for (int k = 0; k < N; ++k) v[it][k] = s_q[k][seg_pad(threadIdx.x * SEG_ITEMS + it)];
    Seg<N> e;
    e.f = h;
#pragma unroll
    for (int k = 0; k < N; ++k) e.v[k] = v[it][k];
    agg = seg_combine(agg, e);
  }
  const Seg<N> ex = block_seg_excl(agg, s_w);
  unsigned long long run[N];
#pragma unroll
  for (int k = 0; k < N; ++k) run[k] = ex.v[k];
  bool seen = ex.f != 0;  // the current segment's head lies in this tile
  // a thread inside one segment, as most are, writes nothing
  if (head == 0u && tail == 0u && !(j0 <= last_valid && last_valid < j0 + SEG_ITEMS)) return;
#pragma unroll
  for (int it = 0; it < SEG_ITEMS; ++it) {
    const uint32_t j = j0 + it;
    if (j >= P.nu) break;
    const bool h = (head >> it) & 1u, t = (tail >> it) & 1u;
#pragma unroll
    for (int k = 0; k < N; ++k) run[k] = h ? v[it][k] : run[k] + v[it][k];
    seen |= h;
    const uint32_t c = key[it];
    if (h) B.cstart[c] = j;
    if (t) {
      B.cend[c] = j + 1;
      if (seen) {
        csum_store_head(B.csum + c, run[0], frame << 1);
        if constexpr (RADAR) B.A[c] = run[N - 1];
      } else {
        atomicAdd(B.S_piece + c, run[0]);
        if constexpr (RADAR) atomicAdd(B.A_piece + c, run[N - 1]);
        B.csum[c].tag = (frame << 1) | 1u;
      }
    } else if (j == last_valid) {
      atomicAdd(B.S_piece + c, run[0]);
      if constexpr (RADAR) atomicAdd(B.A_piece + c, run[N - 1]);
    }
  }
}
template <bool RADAR>
__global__ void __launch_bounds__(SEG_BLOCK) k_segsum(KParams P, DevBufs B) {
  segsum_body<RADAR>(P, B, blockIdx.x);
}

// k_segsum_lidar: k_segsum for a filter without radar likelihood (g == 1), which also sums
// the velocity moment terms of Eq. mean_x, var_x, covar_xy.  With g == 1 the normalised
// weight is w' = mu_UA w with one factor mu_UA = rho_p / S_c per cell, so the moments
// E[v] = sum w' v / rho_p = (mu_UA / rho_p) sum w v follow from sums of the predicted weights,
// one pass earlier than the normalisation.  w v, w v^2, w vx vy are summed per cell as
// compensated double-float sums (exact products, two_sum additions) by the block-wide
// segmented scan; a cell inside the tile leaves its sums in its moment record; a cell spread
// over tiles adds the pieces of S in exact 2^-40 fixed point and leaves its double-float
// moment pieces in per-tile slots, which k_cell adds in tile order.  k_cell applies the
// factor mu_UA / rho_p.
__device__ __forceinline__ void segsum_lidar_body(const KParams &P, const DevBufs &B, uint32_t blk) {
  __shared__ SegQM s_wqm[SEG_BLOCK / 32 + 1];
  __shared__ float s_x[3][SEG_PADDED];  // w, vx, vy in tile order (padded)
  const uint32_t tile = blk, frame = this_frame(B.ctl);
  const uint32_t base = tile * SEG_TILE;
  const uint32_t last_valid = min(base + SEG_TILE, P.nu) - 1u;
  // gather phase, warp-striped, all loads in flight before the stores.  After a resampled
  // frame every predicted weight is p_S w_new, or 0 for a particle that left the grid (the
  // sort carries that flag in the particle index), so only the record is gathered.
  const bool uniform = B.ctl->post_mode == POST_RESAMPLED;
  const float wu = __fmul_rn(P.p_S, B.ctl->w_new);
  // the fixed-point weight: after a resampled frame a weight is wu or 0, so q40(wu) or 0
  const unsigned long long qwu = q40(wu);
  const auto qw = [&](float w) { return uniform ? (w > 0.0f ? qwu : 0ull) : q40(w); };
  uint32_t gi[SEG_ITEMS];
#pragma unroll
  for (int it = 0; it < SEG_ITEMS; ++it) {
    const uint32_t j = base + it * SEG_BLOCK + threadIdx.x;
    gi[it] = j < P.nu ? __ldg(B.perm + j) : 0xffffffffu;
  }
  float4 st[SEG_ITEMS];
  float w[SEG_ITEMS];
#pragma unroll
  for (int it = 0; it < SEG_ITEMS; ++it) {
    st[it] = make_float4(0.f, 0.f, 0.f, 0.f);
    w[it] = 0.0f;
    if (gi[it] != 0xffffffffu) {
      const uint32_t i = gi[it] & ~OUT_OF_GRID;
      st[it] = __ldg(B.As + i);
      w[it] = uniform ? ((gi[it] & OUT_OF_GRID) ? 0.0f : wu) : __ldg(B.Aw + i);
    }
  }
#pragma unroll
  for (int it = 0; it < SEG_ITEMS; ++it) {
    const uint32_t m = it * SEG_BLOCK + threadIdx.x;
    const uint32_t j = base + m;
    if (j < P.nu) {
      B.Os[j] = st[it];
      B.Ow[j] = w[it];
    }
    s_x[0][seg_pad(m)] = w[it];
    s_x[1][seg_pad(m)] = st[it].z;
    s_x[2][seg_pad(m)] = st[it].w;
  }
  __syncthreads();
  // scan phase, blocked: a thread owns ITEMS consecutive positions
  const uint32_t j0 = base + threadIdx.x * SEG_ITEMS;
  uint32_t key[SEG_ITEMS];
  load_run<SEG_ITEMS>(B.key_sorted, j0, P.nu, key, 0xffffffffu);
  const uint32_t kprev = (j0 > 0 && j0 <= P.nu) ? __ldg(B.key_sorted + j0 - 1) : 0xfffffffeu;
  const uint32_t knext = (j0 + SEG_ITEMS < P.nu) ? __ldg(B.key_sorted + j0 + SEG_ITEMS) : 0xfffffffeu;
  uint32_t head = 0, tail = 0;
  SegQM agg;
  agg = seg_zero(agg);
#pragma unroll
  for (int it = 0; it < SEG_ITEMS; ++it) {
    const uint32_t j = j0 + it;
    const bool ok = j < P.nu;
    const uint32_t kp = it == 0 ? kprev : key[it - 1];
    const uint32_t kn = it == SEG_ITEMS - 1 ? knext : key[it + 1];
    const bool h = ok && (j == 0 || key[it] != kp);
    const bool t = ok && (j == P.nu - 1 || key[it] != kn);
    head |= (uint32_t)h << it;
    tail |= (uint32_t)t << it;
    const uint32_t m = seg_pad(threadIdx.x * SEG_ITEMS + it);
    SegQM e;
    e.f = h;
    e.q = qw(s_x[0][m]);
    moment_terms(s_x[0][m], s_x[1][m], s_x[2][m], e.m);
    agg = seg_combine(agg, e);
  }
  const SegQM ex = block_seg_excl(agg, s_wqm);
  unsigned long long rq = ex.q;
  DF rm[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) rm[k] = ex.m[k];
  bool seen = ex.f != 0;  // the current segment's head lies in this tile
  const bool record = (P.flags & 0x4u) != 0u;
  // the running sums are only read at a segment's end (or the tile's last particle): a
  // thread inside one segment, as most are, has nothing more to do
  const bool has_last = j0 <= last_valid && last_valid < j0 + SEG_ITEMS;
  if (tail == 0u && !has_last && !(record && head != 0u)) return;
#pragma unroll
  for (int it = 0; it < SEG_ITEMS; ++it) {
    const uint32_t j = j0 + it;
    if (j >= P.nu) break;
    const bool h = (head >> it) & 1u, t = (tail >> it) & 1u;
    const uint32_t m = seg_pad(threadIdx.x * SEG_ITEMS + it);  // the item's terms again
    const unsigned long long q = qw(s_x[0][m]);
    DF mt[5];
    moment_terms(s_x[0][m], s_x[1][m], s_x[2][m], mt);
    rq = h ? q : rq + q;
#pragma unroll
    for (int k = 0; k < 5; ++k) rm[k] = h ? mt[k] : df_add(rm[k], mt[k]);
    seen |= h;
    const uint32_t c = key[it];
    if (record) {  // explicit cell ranges only for the diagnostic interface
      if (h) B.cstart[c] = j;
      if (t) B.cend[c] = j + 1;
    }
    if (j == last_valid) B.tile_whole[tile] = (!t && !seen) ? 1u : 0u;
    if (t && seen) {  // the whole cell lies in this tile: its head and moment sums
      csum_store_head(B.csum + c, rq, frame << 1);
      cmom_store(B.cmom + c, rm);
    } else if (t || j == last_valid) {  // a piece of a cell spread over several tiles
      // S exactly in fixed point; the moment sums in this tile's slot (0: the cell began in
      // an earlier tile, 1: it continues in a later one), which k_cell adds in tile order
      atomicAdd(B.S_piece + c, rq);
      float *slot = B.Pf + ((size_t)tile * 2u + (seen ? 1u : 0u)) * 10u;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        slot[k] = rm[k].hi;
        slot[5 + k] = rm[k].lo;
      }
      if (seen) B.cross_t1[c] = tile;
      if (t) B.csum[c].tag = (frame << 1) | 1u;
    }
  }
}
__global__ void __launch_bounds__(SEG_BLOCK, 5) k_segsum_lidar(KParams P, DevBufs B) {
  segsum_lidar_body(P, B, blockIdx.x);
}

// ====================================================================================
// k_scan_tiles: inclusive prefix sums of per-tile totals (one block); the grand totals go
// to the control block.  Used for the newborn-mass scan over cell tiles and for the CDF of
// the joint weights over source tiles.
// ====================================================================================
constexpr int SCAN_BLOCK = 1024;

__device__ __forceinline__ float u64_to_f32_approx(unsigned long long x) {
  return __fadd_rn(__fmul_rn((float)(uint32_t)(x >> 32), 0x1p32f), (float)(uint32_t)x);
}

// once per frame, after the CDF total W is known (Alg. 7): the uniform offset
// u = floor(r64 W / 2^64) from one Philox draw, the resampled weight (W 2^-40) / nu rounded
// once from binary64, and a binary32 1/W for the source-range estimates
__device__ void resample_setup(const KParams &P, DevCtl *ctl, unsigned long long Wt) {
  if ((P.flags & 0x2u) != 0u || Wt == 0ull) {
    ctl->u_offset = 0ull;
    ctl->w_new = 0.0f;
    ctl->inv_w = 0.0f;
    ctl->post_mode = POST_DIRECT;
    return;
  }
  ctl->post_mode = POST_RESAMPLED;
  const U4 r = philox(0u, this_frame(ctl), TAG_RESAMPLE, P.seed_lo, P.seed_hi);
  const unsigned long long r64 = ((unsigned long long)r.a << 32) | r.b;
  const unsigned long long u = __umul64hi(r64, Wt);
  ctl->u_offset = u;
  ctl->w_new = (float)((__ull2double_rn(Wt) * 0x1p-40) / (double)P.nu);
  ctl->inv_w = __fdiv_rn(1.0f, u64_to_f32_approx(Wt));
  ctl->th_a = Wt / P.nu;
  ctl->th_b = (uint32_t)(Wt % P.nu);
  ctl->th_c = u / P.nu;
  ctl->th_e = (uint32_t)(u % P.nu);
}

// The systematic rule "output i takes the first source j with Q_j nu > i W + u" reads, for
// integer Q_j, Q_j > theta_i with theta_i = floor((i W + u) / nu); theta_i < 2^64 and is
// exact in 64-bit arithmetic from the split W = a nu + b, u = c nu + e:
// theta_i = i a + c + floor((i b + e) / nu), where i b + e < 2^51.
struct Theta {
  unsigned long long a, c;
  uint32_t b, e, nu;
  float inv_nu;
};
__device__ __forceinline__ Theta theta_of(const DevCtl *ctl, uint32_t nu) {
  return Theta{ctl->th_a, ctl->th_c, ctl->th_b, ctl->th_e, nu, __fdiv_rn(1.0f, (float)nu)};
}
__device__ __forceinline__ unsigned long long theta_at(const Theta &T, uint32_t i, uint32_t *rem = nullptr) {
  const unsigned long long r = (unsigned long long)i * T.b + T.e;
  // floor(r / nu) lies in [0, i]: binary32 estimate (off by a few units at most), then
  // exact corrections, with integer division if the estimate was far off
  const float est = __fmul_rn(u64_to_f32_approx(r), T.inv_nu);
  uint32_t q = !(est > 0.0f) ? 0u : (est >= (float)i ? i : (uint32_t)est);
  int guard = 0;
  while (q > 0u && (unsigned long long)q * T.nu > r && guard < 64) {
    --q;
    ++guard;
  }
  while ((unsigned long long)(q + 1u) * T.nu <= r && guard < 64) {
    ++q;
    ++guard;
  }
  if (guard >= 64) q = (uint32_t)(r / T.nu);
  if (rem) *rem = (uint32_t)(r - (unsigned long long)q * T.nu);  // (i b + e) mod nu
  return (unsigned long long)i * T.a + T.c + q;
}
// #{i in [0, nu) : theta_i < X}, i.e. #{i : i W + u < X nu}: binary32 estimate, exact
// corrections (theta is non-decreasing), bisection if the estimate was far off
__device__ __forceinline__ uint32_t count_theta_below(const Theta &T, unsigned long long X, float inv_w) {
  const uint32_t nu = T.nu;
  if (X <= T.c) return 0u;  // theta_0 = c
  const float est = __fmul_rn(__fmul_rn(u64_to_f32_approx(X - T.c), (float)nu), inv_w);
  uint32_t i = !(est > 0.0f) ? 0u : (est >= (float)nu ? nu : (uint32_t)est);
  int guard = 0;
  while (i > 0u && theta_at(T, i - 1u) >= X && guard < 32) {
    --i;
    ++guard;
  }
  while (i < nu && theta_at(T, i) < X && guard < 32) {
    ++i;
    ++guard;
  }
  if (guard >= 32) {
    uint32_t lo = 0, hi = nu;
    while (lo < hi) {
      const uint32_t mid = lo + (hi - lo) / 2;
      if (theta_at(T, mid) < X) lo = mid + 1; else hi = mid;
    }
    i = lo;
  }
  return i;
}

// SETUP (the joint-weight CDF): the per-frame resampling constants, the tile sums q cleared
// for the next frame once read, and the frame counter advanced (this_frame)
template <bool SETUP>
__device__ __forceinline__ void scan_tiles_body(unsigned long long *q, const uint32_t *__restrict__ n,
                                                uint32_t count, unsigned long long *q_incl, uint32_t *n_incl,
                                                unsigned long long *q_total, uint32_t *n_total, const KParams &P,
                                                DevCtl *ctl) {
  __shared__ unsigned long long s_q[SCAN_BLOCK / 32];
  __shared__ uint32_t s_n[SCAN_BLOCK / 32];
  const uint32_t per = (count + SCAN_BLOCK - 1) / SCAN_BLOCK;
  const uint32_t b = threadIdx.x * per;
  unsigned long long lq = 0ull;
  uint32_t ln = 0u;
  for (uint32_t k = 0; k < per; ++k)
    if (b + k < count) {
      lq += q[b + k];
      if (n) ln += n[b + k];
    }
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long iq = lq;
  uint32_t in = ln;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long tq = __shfl_up_sync(FULL, iq, o);
    const uint32_t tn = __shfl_up_sync(FULL, in, o);
    if (lane >= (uint32_t)o) {
      iq += tq;
      in += tn;
    }
  }
  if (lane == 31) {
    s_q[warp] = iq;
    s_n[warp] = in;
  }
  __syncthreads();
  static_assert(SCAN_BLOCK / 32 == 32, "one warp scans the warp totals");
  if (warp == 0) {  // exclusive scan of the 32 warp totals by one warp
    const unsigned long long vq = s_q[lane];
    const uint32_t vn = s_n[lane];
    unsigned long long xq = vq;
    uint32_t xn = vn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long tq = __shfl_up_sync(FULL, xq, o);
      const uint32_t tn = __shfl_up_sync(FULL, xn, o);
      if (lane >= (uint32_t)o) {
        xq += tq;
        xn += tn;
      }
    }
    s_q[lane] = xq - vq;
    s_n[lane] = xn - vn;
    if (lane == 31) {
      *q_total = xq;
      if (n_total) *n_total = xn;
      if constexpr (SETUP) {
        resample_setup(P, ctl, xq);
        ctl->frame += 1u;  // the frame's last reader of its number is done
      }
    }
  }
  __syncthreads();
  unsigned long long rq = s_q[warp] + iq - lq;
  uint32_t rn = s_n[warp] + in - ln;
  for (uint32_t k = 0; k < per; ++k)
    if (b + k < count) {
      rq += q[b + k];
      if constexpr (SETUP) q[b + k] = 0ull;  // for the next frame's atomics
      q_incl[b + k] = rq;
      if (n) {
        rn += n[b + k];
        n_incl[b + k] = rn;
      }
    }
}
template <bool SETUP>
__global__ void __launch_bounds__(SCAN_BLOCK)
    k_scan_tiles(unsigned long long *q, const uint32_t *__restrict__ n, uint32_t count,
                 unsigned long long *q_incl, uint32_t *n_incl, unsigned long long *q_total,
                 uint32_t *n_total, KParams P, DevCtl *ctl) {
  scan_tiles_body<SETUP>(q, n, count, q_incl, n_incl, q_total, n_total, P, ctl);
}

// ====================================================================================
// k_cell (Alg. 3 + the cell half of Alg. 4): per cell the predicted occupied mass
// min(S, 1), the free-mass prediction, Dempster's rule with the measurement BBA, the
// newborn / persistent split and the normalisers mu_A, mu_UA.  Each tile lists, in cell
// order, its cells with newborn mass together with the tile-local inclusive prefix of the
// fixed-point newborn masses; k_scan_tiles then scans the tile totals.
// ====================================================================================
constexpr int CELL_BLOCK = 256, CELL_ITEMS = 2, CELL_TILE = CELL_BLOCK * CELL_ITEMS;

__device__ __forceinline__ void cell_update(const KParams &P, float mp, float mFprev, float zO, float zF,
                                            float &mO, float &mF, float &rb) {
  const float mFp = fminf(__fmul_rn(P.alpha, mFprev), __fsub_rn(1.0f, mp));
  const float mT = __fsub_rn(__fsub_rn(1.0f, mp), mFp);
  const float zT = __fsub_rn(__fsub_rn(1.0f, zO), zF);
  const float K = __fadd_rn(__fmul_rn(mp, zF), __fmul_rn(mFp, zO));
  const float den = __fsub_rn(1.0f, K);
  if (den < 1e-6f) {
    mO = mp;
    mF = mFp;
  } else {
    const float nO = __fadd_rn(__fadd_rn(__fmul_rn(mp, zO), __fmul_rn(mp, zT)), __fmul_rn(mT, zO));
    const float nF = __fadd_rn(__fadd_rn(__fmul_rn(mFp, zF), __fmul_rn(mFp, zT)), __fmul_rn(mT, zF));
    mO = __fdiv_rn(nO, den);
    mF = __fdiv_rn(nF, den);
  }
  rb = 0.0f;
  if (zO > 0.0f) {
    const float pb = __fmul_rn(P.p_B, __fsub_rn(1.0f, mp));
    const float d = __fadd_rn(mp, pb);
    if (d > 0.0f) rb = __fdiv_rn(__fmul_rn(mO, pb), d);
    if (rb > mO) rb = mO;
  }
}

template <bool RADAR>
__device__ __forceinline__ void cell_body(const KParams &P, const DevBufs &B, uint32_t blk) {
  __shared__ unsigned long long s_wq[CELL_BLOCK / 32 + 1];
  __shared__ uint32_t s_wn[CELL_BLOCK / 32 + 1];
  const uint32_t tile = blk, frame = this_frame(B.ctl);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long qin[CELL_ITEMS];
  uint32_t nex[CELL_ITEMS];
  bool has[CELL_ITEMS];
  unsigned long long wq = 0ull;  // running sums of this warp, in cell order
  uint32_t wn = 0u;
  // all loads of the thread's cells first (independent, in flight together)
  uint32_t tgs[CELL_ITEMS];
  float mFs[CELL_ITEMS], zOs[CELL_ITEMS], zFs[CELL_ITEMS];
  unsigned long long Ss[CELL_ITEMS];
  const bool full = !RADAR && (P.flags & FLAG_FULL) != 0u;  // the PHD/MIB filter of Sect. VI
#pragma unroll
  for (int it = 0; it < CELL_ITEMS; ++it) {
    const uint32_t c = tile * CELL_TILE + warp * (32 * CELL_ITEMS) + it * 32 + lane;
    const bool in = c < P.C;
    const uint4 h = in ? *reinterpret_cast<const uint4 *>(B.csum + c) : make_uint4(0u, 0u, 0u, 0u);
    Ss[it] = ((unsigned long long)h.y << 32) | h.x;
    tgs[it] = h.z;
    mFs[it] = in ? B.mF_in[c] : 0.0f;
    zOs[it] = in ? B.zO[c] : 0.0f;
    zFs[it] = in ? B.zF[c] : 0.0f;
  }
#pragma unroll
  for (int it = 0; it < CELL_ITEMS; ++it) {
    const uint32_t c = tile * CELL_TILE + warp * (32 * CELL_ITEMS) + it * 32 + lane;
    const bool occ = c < P.C && (tgs[it] >> 1) == frame;
    if (!occ) Ss[it] = 0ull;
    if (occ && (tgs[it] & 1u)) {
      Ss[it] = atomicExch(B.S_piece + c, 0ull);  // all pieces are in; clear for the next frame
      B.csum[c].S = Ss[it];
    }
  }
#pragma unroll
  for (int it = 0; it < CELL_ITEMS; ++it) {
    const uint32_t c = tile * CELL_TILE + warp * (32 * CELL_ITEMS) + it * 32 + lane;
    unsigned long long qb = 0ull;
    if (c < P.C) {
      const uint32_t tg = tgs[it];
      const bool occ = (tg >> 1) == frame;
      const bool cross = occ && (tg & 1u);
      const unsigned long long S = Ss[it];
      const float Sf = fx40_to_f(S);
      const float mp = fminf(Sf, 1.0f);
      float mO, mF, rb, rp, alloc, muU;
      float muA = 0.0f, pa = 0.0f;
      if (full) {
        // predicted Bernoulli RFS: persistent existence r_p = min(S, 1) (the weights of a cell
        // whose sum exceeds 1 are scaled to sum 1), newborn r_b = p_B (1 - r_p) (Eq.
        // pred_birth_prob); the Bernoulli update (Eq. filter_update, normalization_empty,
        // normalization_meas) with the single-object likelihood 1 multiplies every particle
        // weight of the cell by one factor f (Eq. updateParticleWeightsUnnormalized,
        // applyNormalization, updateParticleWeightsEmpty)
        const float rbp = __fmul_rn(P.p_B, __fsub_rn(1.0f, mp));
        const float r = __fadd_rn(mp, rbp);
        const float omr = __fsub_rn(1.0f, r);
        const float ptp = zFs[it], pfp = B.zv[c];
        float f;
        if (zOs[it] != 0.0f) {
          const float pa_ = B.pA[c], pc = B.sgv[c];
          const float gam = __fadd_rn(pa_, __fmul_rn(__fsub_rn(1.0f, pa_), pc));
          const float num = __fmul_rn(ptp, gam);
          const float Nz = __fadd_rn(__fmul_rn(__fmul_rn(pfp, pc), omr), __fmul_rn(num, r));
          f = __fdiv_rn(num, Nz);
        } else {
          const float a = __fsub_rn(1.0f, ptp);
          const float Ne = __fadd_rn(__fmul_rn(a, r), __fmul_rn(__fsub_rn(1.0f, pfp), omr));
          f = __fdiv_rn(a, Ne);
        }
        rp = __fmul_rn(f, mp);
        rb = __fmul_rn(f, rbp);
        mO = __fadd_rn(rp, rb);       // posterior existence = occupancy probability
        mF = __fsub_rn(1.0f, mO);
        alloc = rbp;                  // newborn slots follow the predicted newborn existence
        muA = f;                      // newborn weights f r_b / n (k_birth_prep)
        B.rb_pred[c] = rbp;
        B.pO[c] = mO;
        muU = (S > 0ull) ? (Sf > 1.0f ? __fdiv_rn(f, Sf) : f) : 0.0f;
      } else {
        cell_update(P, mp, mFs[it], zOs[it], zFs[it], mO, mF, rb);
        rp = __fsub_rn(mO, rb);
        alloc = rb;
        B.pO[c] = __fadd_rn(mO, __fmul_rn(0.5f, __fsub_rn(__fsub_rn(1.0f, mO), mF)));
        muU = (S > 0ull) ? __fdiv_rn(rp, Sf) : 0.0f;
      }
      B.muU[c] = muU;
      // (m_pred itself is not stored: the diagnostic read recomputes it from S, k_mpred)
      B.mO[c] = mO;
      B.mF[c] = mF;
      B.rho_b[c] = rb;
      B.rho_p[c] = rp;
      if constexpr (RADAR) {
        unsigned long long A = 0ull;
        if (cross) {
          A = atomicExch(B.A_piece + c, 0ull);
          B.A[c] = A;
        } else if (occ) {
          A = B.A[c];
        }
        if (A > 0ull) {
          muA = __fdiv_rn(rp, fx40_to_f(A));
          pa = B.pA[c];
        }
        B.paeff[c] = pa;
      }
      // mu_A: read by the radar normalisation and the PHD/MIB newborn weights; a lidar DS
      // filter's stays 0 from the workspace's initialisation
      if (RADAR || full) B.muA[c] = muA;
      if constexpr (!RADAR) {  // moments of the lidar filter (see k_segsum_lidar)
        // E[v] = sum w' v / rho_p with w' = mu_UA w: the compensated sums of w v, ... times
        // mu_UA / rho_p in double-float (Eq. mean_x, var_x, covar_xy)
        float o[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (occ && rp > 0.0f && muU > 0.0f) {
          DF mm[5];
          if (cross) {  // the cell's pieces in tile order: first, whole tiles, last
            uint32_t t = B.cross_t1[c];
            const float *first = B.Pf + ((size_t)t * 2u + 1u) * 10u;
#pragma unroll
            for (int k = 0; k < 5; ++k) mm[k] = DF{first[k], first[5 + k]};
            for (++t; t < P.tiles_seg; ++t) {
              const float *pc = B.Pf + (size_t)t * 20u;
#pragma unroll
              for (int k = 0; k < 5; ++k) mm[k] = df_add(mm[k], DF{pc[k], pc[5 + k]});
              if (!B.tile_whole[t]) break;
            }
          } else {  // finished by the segment pass
            cmom_load(B.cmom + c, mm);
          }
          moments_scaled(mm, muU, rp, o);
        }
        moments_store(B, c, o);
      } else if (!occ) {
        float z[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        moments_store(B, c, z);
      }
      qb = q40(alloc);
    }
    has[it] = qb > 0ull;
    // position among the warp's cells with newborn mass (ballot) and the inclusive prefix
    // of their masses; cells with newborn mass are sparse, so most warps skip the scan
    const uint32_t hb = __ballot_sync(FULL, has[it]);
    nex[it] = wn + __popc(hb & lanemask_lt());
    qin[it] = wq;
    if (hb != 0u) {  // warp-uniform
      unsigned long long sq = qb;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long tq = __shfl_up_sync(FULL, sq, o);
        if (lane >= (uint32_t)o) sq += tq;
      }
      qin[it] = wq + sq;
      wq += __shfl_sync(FULL, sq, 31);
    }
    wn += __popc(hb);
  }
  if (lane == 0) {
    s_wq[warp] = wq;
    s_wn[warp] = wn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long rq = 0ull;
    uint32_t rn = 0u;
    for (int w = 0; w < CELL_BLOCK / 32; ++w) {
      const unsigned long long tq = s_wq[w];
      const uint32_t tn = s_wn[w];
      s_wq[w] = rq;
      s_wn[w] = rn;
      rq += tq;
      rn += tn;
    }
    B.tile_q[tile] = rq;
    B.tile_n[tile] = rn;
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < CELL_ITEMS; ++it) {
    if (has[it]) {
      const uint32_t c = tile * CELL_TILE + warp * (32 * CELL_ITEMS) + it * 32 + lane;
      const uint32_t pos = tile * CELL_TILE + s_wn[warp] + nex[it];
      B.bl_cell[pos] = c;
      B.bl_R[pos] = s_wq[warp] + qin[it];
    }
  }
}
template <bool RADAR>
__global__ void __launch_bounds__(CELL_BLOCK) k_cell(KParams P, DevBufs B) {
  cell_body<RADAR>(P, B, blockIdx.x);
}

// ====================================================================================
// k_birth (Alg. 5): cell c owns the newborn slots [floor(nu_b R_{c-1}/R), floor(nu_b R_c/R))
// of the fixed-point scan R of the newborn masses; nu_A = round(n p_A) of them form the
// associated set (Eq. assoc_relation, assoc_sum), with weights Eq. weights_associated /
// weights_unassociated.  The exact slot arithmetic is done once per birth cell
// (k_birth_prep); each slot then only searches first-slot tables.
// ====================================================================================
constexpr int BIRTH_BLOCK = 256;

__device__ __forceinline__ void birth_init(const KParams &P, const DevBufs &B, uint32_t slot,
                                           uint32_t c, bool assoc, float w, float zv, float sg,
                                           uint32_t frame, bool record) {
  const U4 r = philox(slot, frame, TAG_BIRTH, P.seed_lo, P.seed_hi);
  const float col = (float)(c % (uint32_t)P.W), row = (float)(c / (uint32_t)P.W);
  const float x = __fmul_rn(__fadd_rn(col, u01_co(r.a)), P.s);
  const float y = __fmul_rn(__fadd_rn(row, u01_co(r.b)), P.s);
  float n0, n1;
  gauss2(r.c, r.d, n0, n1);
  float vx, vy;
  if (assoc) {
    const float dx = __fsub_rn(x, P.sensor_x), dy = __fsub_rn(y, P.sensor_y);
    const float rr = __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
    float ex = 1.0f, ey = 0.0f;
    if (rr > 0.0f) {
      ex = __fdiv_rn(dx, rr);
      ey = __fdiv_rn(dy, rr);
    }
    const float vr = __fadd_rn(zv, __fmul_rn(sg, n0));
    const float vt = __fmul_rn(P.sigma_B, n1);
    vx = __fsub_rn(__fmul_rn(vr, ex), __fmul_rn(vt, ey));
    vy = __fadd_rn(__fmul_rn(vr, ey), __fmul_rn(vt, ex));
  } else {
    vx = __fmul_rn(P.sigma_B, n0);
    vy = __fmul_rn(P.sigma_B, n1);
  }
  B.bs[slot] = make_float4(x, y, vx, vy);
  B.bw[slot] = w;
  if (record) {
    B.bcell[slot] = c;
    B.bassoc[slot] = assoc ? 1u : 0u;
  }
}

// k_birth_prep: per birth cell (list entry) its first slot floor(nu_b R_{c-1} / R), the
// associated count nu_A = round(n p_A) and the two newborn weights, written to one list in
// cell order (entry G = birth cells of earlier tiles + position in the tile); and, for each
// block of BIRTH_SLOTS slots, the entry that owns the block's first slot.  One block per
// cell tile.
constexpr int BIRTH_SLOTS = 512, BIRTH_CACHE = 2048;
constexpr int BPREP_BLOCK = 128;  // a cell tile's list holds a few birth cells on average

template <bool RADAR>
__device__ __forceinline__ void birth_prep_body(const KParams &P, const DevBufs &B, uint32_t blk) {
  const unsigned long long R = B.ctl->R_total;
  if (R == 0ull) return;
  const uint32_t T = blk;
  const unsigned long long Tex = T > 0u ? B.tile_qin[T - 1u] : 0ull;
  const uint32_t G0 = T > 0u ? B.tile_nin[T - 1u] : 0u;
  if (T == P.tiles_cell - 1u && threadIdx.x == 0) B.bl_first[B.tile_nin[T]] = P.nu_b;  // sentinel
  const uint32_t cnt = B.tile_n[T];
  for (uint32_t e = threadIdx.x; e < cnt; e += BPREP_BLOCK) {
    const size_t pos = (size_t)T * CELL_TILE + e;
    const uint32_t c = B.bl_cell[pos];
    const unsigned long long Rin = Tex + B.bl_R[pos];
    const unsigned long long Rex = Tex + (e > 0u ? B.bl_R[pos - 1] : 0ull);
    const uint32_t first = floor_muldiv(P.nu_b, Rex, R);
    const uint32_t last = floor_muldiv(P.nu_b, Rin, R);
    const uint32_t n = last > first ? last - first : 0u;
    const bool full = !RADAR && (P.flags & FLAG_FULL) != 0u;
    const float rb = full ? B.rb_pred[c] : B.rho_b[c];
    const float pA = RADAR ? B.pA[c] : 0.0f;
    uint32_t nA = (uint32_t)__fadd_rn(__fmul_rn((float)n, pA), 0.5f);
    if (nA > n) nA = n;
    const uint32_t nUA = n - nA;
    float wA = 0.0f, wUA = 0.0f;
    if (nA > 0u && nUA > 0u) {
      wA = __fdiv_rn(__fmul_rn(pA, rb), (float)nA);
      wUA = __fdiv_rn(__fmul_rn(__fsub_rn(1.0f, pA), rb), (float)nUA);
    } else if (n > 0u) {
      wA = wUA = __fdiv_rn(rb, (float)n);
    }
    if (full) wA = wUA = __fmul_rn(B.muA[c], wUA);  // predicted r_b / n, updated by f
    const uint32_t G = G0 + e;
    B.bl_first[G] = first;
    B.bl_gcell[G] = c;
    B.bl_nA[G] = nA;
    B.bl_wA[G] = wA;
    B.bl_wUA[G] = wUA;
    // slot blocks whose first slot lies in [first, last)
    for (uint32_t blk = (first + BIRTH_SLOTS - 1u) / BIRTH_SLOTS; blk * BIRTH_SLOTS < last; ++blk)
      B.birth_block_entry[blk] = G;
  }
}
template <bool RADAR>
__global__ void __launch_bounds__(BPREP_BLOCK) k_birth_prep(KParams P, DevBufs B) {
  birth_prep_body<RADAR>(P, B, blockIdx.x);
}

constexpr int NORM_TILE_ = 2048;  // the resampling tile (NORM_TILE, defined with k_normalise)
static_assert(BIRTH_SLOTS <= NORM_TILE_, "a newborn block spans at most two resampling tiles");

// add a block's newborn weight sums q0 (tile t0) and q1 (tile t1 = t0 + 1, if any) to the
// resampling tiles' joint-weight sums (exact 64-bit atomics: the order of the additions does
// not matter)
__device__ __forceinline__ void birth_tile_sums(const DevBufs &B, unsigned long long q0, unsigned long long q1,
                                                uint32_t t0, uint32_t t1) {
  __shared__ unsigned long long s_q[2][BIRTH_BLOCK / 32];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    q0 += __shfl_xor_sync(FULL, q0, o);
    q1 += __shfl_xor_sync(FULL, q1, o);
  }
  if (lane == 0) {
    s_q[0][warp] = q0;
    s_q[1][warp] = q1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0ull, b = 0ull;
    for (int w = 0; w < BIRTH_BLOCK / 32; ++w) {
      a += s_q[0][w];
      b += s_q[1][w];
    }
    if (a) atomicAdd(B.cdf_tile + t0, a);
    if (t1 != t0 && b) atomicAdd(B.cdf_tile + t1, b);
  }
}

// k_birth: a block makes the newborns of BIRTH_SLOTS consecutive slots.  Its slots belong to
// the entries from the one owning its first slot to the one owning the next block's first
// slot; it caches those entries' first slots in shared memory (at most BIRTH_CACHE of them),
// and each slot finds its entry (the last one whose first slot is <= the slot) by bisection
// there.
template <bool RADAR>
__device__ __forceinline__ void birth_body(const KParams &P, const DevBufs &B, uint32_t blk) {
  __shared__ uint32_t s_first[BIRTH_CACHE + 1];
  const uint32_t frame = this_frame(B.ctl);
  const unsigned long long R = B.ctl->R_total;
  const bool record = (P.flags & 0x4u) != 0u;
  const uint32_t s0 = blk * BIRTH_SLOTS;
  const uint32_t s1 = min(s0 + BIRTH_SLOTS, P.nu_b);
  if (s0 >= s1) return;  // block-uniform (no newborn slots at all)
  if (R == 0ull) {
    // no newborn mass anywhere: weight 0, cell = slot mod C
    for (uint32_t s = s0 + threadIdx.x; s < s1; s += BIRTH_BLOCK)
      birth_init(P, B, s, s % P.C, false, 0.0f, 0.0f, 1.0f, frame, record);
    return;
  }
  const uint32_t nE = B.ctl->n_birth_cells;
  const uint32_t G0 = B.birth_block_entry[blk];
  const uint32_t Glast = s1 < P.nu_b ? B.birth_block_entry[blk + 1] : nE - 1u;
  // entries G0 .. G0 + ncache - 1, and bl_first[G0 + ncache] (<= the sentinel at nE) after them
  const uint32_t ncache = min((uint32_t)BIRTH_CACHE, Glast - G0 + 1u);
  for (uint32_t k = threadIdx.x; k <= ncache; k += BIRTH_BLOCK) s_first[k] = __ldg(B.bl_first + G0 + k);
  __syncthreads();
  const uint32_t cached_end = s_first[ncache];  // first slot after the cached entries
  // entry of each of the thread's slots, then all entry gathers, then the draws
  constexpr int PER = BIRTH_SLOTS / BIRTH_BLOCK;
  uint32_t G[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const uint32_t s = s0 + r * BIRTH_BLOCK + threadIdx.x;
    G[r] = 0u;
    if (s >= s1) continue;
    if (s < cached_end) {
      uint32_t a = 0, b = ncache - 1u;
      while (a < b) {
        const uint32_t mid = (a + b + 1u) >> 1;
        if (s_first[mid] <= s) a = mid; else b = mid - 1u;
      }
      G[r] = G0 + a;
    } else {  // beyond the cache (many entries without slots in this block): global bisection
      uint32_t a = G0 + ncache, b = nE - 1u;
      while (a < b) {
        const uint32_t mid = (a + b + 1u) >> 1;
        if (__ldg(B.bl_first + mid) <= s) a = mid; else b = mid - 1u;
      }
      G[r] = a;
    }
  }
  uint32_t cell[PER];
  bool assoc[PER];
  float wb[PER], zv[PER], sg[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const uint32_t s = s0 + r * BIRTH_BLOCK + threadIdx.x;
    cell[r] = 0u;
    assoc[r] = false;
    wb[r] = 0.0f;
    zv[r] = 0.0f;
    sg[r] = 1.0f;
    if (s >= s1) continue;
    cell[r] = __ldg(B.bl_gcell + G[r]);
    assoc[r] = s - __ldg(B.bl_first + G[r]) < __ldg(B.bl_nA + G[r]);
    wb[r] = assoc[r] ? __ldg(B.bl_wA + G[r]) : __ldg(B.bl_wUA + G[r]);
    if constexpr (RADAR) {
      zv[r] = __ldg(B.zv + cell[r]);
      sg[r] = __ldg(B.sgv + cell[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const uint32_t s = s0 + r * BIRTH_BLOCK + threadIdx.x;
    if (s < s1) birth_init(P, B, s, cell[r], assoc[r], wb[r], zv[r], sg[r], frame, record);
  }
  // the newborn part of the resampling tiles' joint-weight sums: slot s is joint source
  // nu + s; this block's slots lie in at most two tiles (BIRTH_SLOTS <= NORM_TILE)
  const uint32_t t_first = (P.nu + s0) / NORM_TILE_;
  unsigned long long q0 = 0ull, q1 = 0ull;
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const uint32_t s = s0 + r * BIRTH_BLOCK + threadIdx.x;
    if (s >= s1) continue;
    const unsigned long long q = q40(wb[r]);
    if ((P.nu + s) / NORM_TILE_ == t_first) q0 += q; else q1 += q;
  }
  birth_tile_sums(B, q0, q1, t_first, (P.nu + s1 - 1u) / NORM_TILE_);
}
template <bool RADAR>
__global__ void __launch_bounds__(BIRTH_BLOCK) k_birth(KParams P, DevBufs B) {
  birth_body<RADAR>(P, B, blockIdx.x);
}

// ====================================================================================
// k_normalise (Alg. 4): over the joint source index space (persistent particles in sorted
// order, read contiguously from the sorted copy, then newborn slots):
//   w' = p_A mu_A g w + (1 - p_A) mu_UA w   (Eq. DSnormalization; lidar cells: mu_UA w),
//   and the persistent part of the tile sums of q40 of the joint weights for the resampling
//   CDF (k_birth adds the newborn part).  The grid covers the persistent sources only.  The
//   radar filter's velocity moments (Alg. 6) follow in k_rmsum and k_moments.
// ====================================================================================
constexpr int NORM_BLOCK = 256, NORM_ITEMS = 8, NORM_TILE = NORM_BLOCK * NORM_ITEMS;
static_assert(NORM_TILE == NORM_TILE_, "the newborn kernel's resampling tile");
static_assert(NORM_BLOCK == SEG_BLOCK, "k_normalise shares the segment pass's block scan");

// shared-memory index of a thread's item, padded by one element per NORM_ITEMS so that a
// warp reading its threads' item k hits distinct banks
__device__ __forceinline__ uint32_t norm_pad(uint32_t m) { return m + m / NORM_ITEMS; }
constexpr int NORM_PADDED = NORM_TILE + NORM_TILE / NORM_ITEMS;

// the radar filter's normalisation: w' per persistent source and the tile's part of the
// joint quantised weights (the velocity moments follow in k_rmsum)
template <bool RADAR>
__device__ __forceinline__ void normalise_body(const KParams &P, const DevBufs &B, uint32_t blk) {
  __shared__ unsigned long long s_red[NORM_BLOCK / 32];
  const uint32_t tile = blk;
  const uint32_t j0 = tile * NORM_TILE + threadIdx.x * NORM_ITEMS;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long qsum = 0ull;
  if (tile * NORM_TILE < P.nu) {  // block-uniform
    uint32_t key[NORM_ITEMS];
    float ws[NORM_ITEMS], gs[NORM_ITEMS];
    load_run<NORM_ITEMS>(B.key_sorted, j0, P.nu, key, 0xffffffffu);
    load_runf<NORM_ITEMS>(B.Ow, j0, P.nu, ws);
    // the radar likelihood g of each particle, left in wn by k_segsum (for every particle of
    // a cell with p_A > 0, which includes every cell with an effective p_A > 0)
    if (RADAR) load_runf<NORM_ITEMS>(B.wn, j0, P.nu, gs);
    // per-cell factors of all items before any arithmetic (independent loads in flight)
    float cmu[NORM_ITEMS];
#pragma unroll
    for (int it = 0; it < NORM_ITEMS; ++it) cmu[it] = j0 + it < P.nu ? __ldg(B.muU + key[it]) : 0.0f;
    float wnv[NORM_ITEMS];
#pragma unroll
    for (int it = 0; it < NORM_ITEMS; ++it) {
      wnv[it] = 0.0f;
      if (j0 + it < P.nu) {
        const uint32_t c = key[it];
        const float w = ws[it];
        const float muU = cmu[it];
        float wn;
        const float pa = RADAR ? __ldg(B.paeff + c) : 0.0f;
        if (RADAR && pa > 0.0f) {
          const float g = gs[it];
          const float a = __fmul_rn(__fmul_rn(__fmul_rn(pa, __ldg(B.muA + c)), g), w);
          const float b = __fmul_rn(__fmul_rn(__fsub_rn(1.0f, pa), muU), w);
          wn = __fadd_rn(a, b);
        } else {
          wn = __fmul_rn(muU, w);
        }
        wnv[it] = wn;
        qsum += q40(wn);
      }
    }
    store_run<NORM_ITEMS>(B.wn, j0, P.nu, wnv);
  }
  // this tile's persistent part of the joint quantised weights (k_birth adds the newborn
  // part; k_scan_tiles turns the tile sums into the CDF)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qsum += __shfl_xor_sync(FULL, qsum, o);
  if (lane == 0) s_red[warp] = qsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tsum = 0ull;
    for (int w = 0; w < NORM_BLOCK / 32; ++w) tsum += s_red[w];
    atomicAdd(B.cdf_tile + tile, tsum);
    if (tile == 0u) B.ctl->frame_mom = this_frame(B.ctl);  // for k_moments
  }
}
template <bool RADAR>
__global__ void __launch_bounds__(NORM_BLOCK) k_normalise(KParams P, DevBufs B) {
  normalise_body<RADAR>(P, B, blockIdx.x);
}

// k_rmsum (radar filter, after k_normalise, beside the CDF scan and the resampling: nothing
// later in the frame reads the moments): the velocity moments of the persistent particles
// per cell (Eq. mean_x, var_x, covar_xy) from the normalised weights w' the normalisation
// left in wn.  The terms w' v, w' v^2, w' vx vy are formed as exact double-float products
// and summed by the block's segmented scan with compensated additions; a cell inside the
// tile leaves its sums in its moment record; a cell spread over several tiles adds its
// pieces, divided by rho_p, in exact 2^-40 fixed point with integer atomics; k_moments
// finishes both.
__device__ __forceinline__ void rmsum_body(const KParams &P, const DevBufs &B, uint32_t blk) {
  __shared__ SegMom s_w[NORM_BLOCK / 32 + 1];
  __shared__ float s_t[3][NORM_PADDED];  // w', vx, vy of the tile's items, for the tail pass
  const uint32_t tile = blk;
  if (tile * NORM_TILE >= P.nu) return;  // block-uniform
  const uint32_t j0 = tile * NORM_TILE + threadIdx.x * NORM_ITEMS;
  uint32_t key[NORM_ITEMS];
  uint32_t head = 0, tail = 0;
  SegMom agg;
  agg = seg_zero(agg);
  {
    float wnv[NORM_ITEMS];
    load_run<NORM_ITEMS>(B.key_sorted, j0, P.nu, key, 0xffffffffu);
    load_runf<NORM_ITEMS>(B.wn, j0, P.nu, wnv);
    float mvx[NORM_ITEMS], mvy[NORM_ITEMS];
#pragma unroll
    for (int it = 0; it < NORM_ITEMS; ++it) {
      const float4 st = j0 + it < P.nu ? __ldg(B.Os + j0 + it) : make_float4(0.f, 0.f, 0.f, 0.f);
      mvx[it] = st.z;
      mvy[it] = st.w;
    }
    const uint32_t kprev = (j0 > 0 && j0 <= P.nu) ? __ldg(B.key_sorted + j0 - 1) : 0xfffffffeu;
    const uint32_t knext = (j0 + NORM_ITEMS < P.nu) ? __ldg(B.key_sorted + j0 + NORM_ITEMS) : 0xfffffffeu;
#pragma unroll
    for (int it = 0; it < NORM_ITEMS; ++it) {
      const uint32_t j = j0 + it;
      const bool ok = j < P.nu;
      const uint32_t kp = it == 0 ? kprev : key[it - 1];
      const uint32_t kn = it == NORM_ITEMS - 1 ? knext : key[it + 1];
      const bool h = ok && (j == 0 || key[it] != kp);
      const bool t = ok && (j == P.nu - 1 || key[it] != kn);
      head |= (uint32_t)h << it;
      tail |= (uint32_t)t << it;
      SegMom e;
      e.f = h;
      moment_terms(wnv[it], mvx[it], mvy[it], e.m);
      agg = seg_combine(agg, e);
      const uint32_t m = norm_pad(threadIdx.x * NORM_ITEMS + it);
      s_t[0][m] = wnv[it];
      s_t[1][m] = mvx[it];
      s_t[2][m] = mvy[it];
    }
  }
  // segmented compensated moment sums within the tile
  const SegMom ex = block_seg_excl(agg, s_w);
  const uint32_t last_valid = min(tile * NORM_TILE + NORM_TILE, P.nu) - 1u;
  DF run[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) run[k] = ex.m[k];
  bool seen = ex.f != 0;
  // the running sums are only read at a segment's end or the tile's last particle
  if (tail == 0u && !(j0 <= last_valid && last_valid < j0 + NORM_ITEMS)) return;
#pragma unroll
  for (int it = 0; it < NORM_ITEMS; ++it) {
    const uint32_t j = j0 + it;
    if (j >= P.nu) break;
    const bool h = (head >> it) & 1u, t = (tail >> it) & 1u;
    const uint32_t mi = norm_pad(threadIdx.x * NORM_ITEMS + it);
    DF m[5];
    moment_terms(s_t[0][mi], s_t[1][mi], s_t[2][mi], m);
#pragma unroll
    for (int k = 0; k < 5; ++k) run[k] = h ? m[k] : df_add(run[k], m[k]);
    seen |= h;
    if (!t && j != last_valid) continue;
    const uint32_t c = key[it];
    if (t && seen) {  // the cell lies in this tile: its raw sums, finished by k_moments
      cmom_store(B.cmom + c, run);
      continue;
    }
    // a piece of a cell spread over several tiles: its sums divided by rho_p, accumulated
    // exactly in fixed point (|E[v]| <= max |v|, so the 2^-40 quanta are absolute errors)
    const float rp = __ldg(B.rho_p + c);
    if (!(rp > 0.0f)) continue;
    const size_t Cs = P.C;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const DF e = df_div_f(run[k], rp);
      atomicAdd(B.Mx + k * Cs + c, q40s(e.hi) + q40s(e.lo));
    }
  }
}
__global__ void __launch_bounds__(NORM_BLOCK, 4) k_rmsum(KParams P, DevBufs B) { rmsum_body(P, B, blockIdx.x); }

// k_moments (radar filter, after k_rmsum): the velocity moments of every cell with
// particles this frame from its compensated sums of w' v, ... divided by rho_p (a cell
// inside one normalisation tile) or from its exact fixed-point pieces (a cell spread over
// several; read and cleared for the next frame); 0 where rho_p = 0.
__device__ __forceinline__ void moments_body(const KParams &P, const DevBufs &B, uint32_t blk, uint32_t nblk) {
  const uint32_t frame = B.ctl->frame_mom;  // the counter itself may have advanced already
  const size_t Cs = P.C;
  for (uint32_t c = blk * blockDim.x + threadIdx.x; c < P.C; c += nblk * blockDim.x) {
    const uint32_t tag = B.csum[c].tag;
    if ((tag >> 1) != frame || frame == 0u) continue;  // no particles: zeros from k_cell
    const uint32_t a = B.cstart[c], e = B.cend[c];
    const bool whole = a / NORM_TILE == (e - 1u) / NORM_TILE;
    const float rp = B.rho_p[c];
    float o[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (whole) {
      if (rp > 0.0f) {
        DF m[5];
        cmom_load(B.cmom + c, m);
        moments_scaled(m, 1.0f, rp, o);
      }
    } else {
      DF E[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) E[k] = fx40s_to_df(atomicExch(B.Mx + k * Cs + c, 0ull));
      if (rp > 0.0f) moments_of_expectations(E, o);
    }
    moments_store(B, c, o);
  }
}
__global__ void __launch_bounds__(256) k_moments(KParams P, DevBufs B) { moments_body(P, B, blockIdx.x, gridDim.x); }

// k_normalise_lidar: the lidar filter's normalisation (Eq. DSnormalization with g == 1:
// w' = mu_UA w, Alg. 4) over the persistent sources and their part of the tile sums of the
// joint quantised weights; its moments were summed in k_segsum_lidar.
__device__ __forceinline__ void normalise_lidar_body(const KParams &P, const DevBufs &B, uint32_t blk) {
  __shared__ unsigned long long s_red[NORM_BLOCK / 32];
  const uint32_t tile = blk;
  const uint32_t j0 = tile * NORM_TILE + threadIdx.x * NORM_ITEMS;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long qsum = 0ull;
  if (tile * NORM_TILE < P.nu) {  // block-uniform
    uint32_t key[NORM_ITEMS];
    float ws[NORM_ITEMS], cmu[NORM_ITEMS], wn[NORM_ITEMS];
    load_run<NORM_ITEMS>(B.key_sorted, j0, P.nu, key, 0xffffffffu);
    load_runf<NORM_ITEMS>(B.Ow, j0, P.nu, ws);
#pragma unroll
    for (int it = 0; it < NORM_ITEMS; ++it) cmu[it] = j0 + it < P.nu ? __ldg(B.muU + key[it]) : 0.0f;
    unsigned long long qprev = 0ull;
#pragma unroll
    for (int it = 0; it < NORM_ITEMS; ++it) {  // neighbours mostly share a cell and so a weight
      wn[it] = __fmul_rn(cmu[it], ws[it]);
      qprev = (it > 0 && wn[it] == wn[it - 1]) ? qprev : q40(wn[it]);
      qsum += qprev;
    }
    store_run<NORM_ITEMS>(B.wn, j0, P.nu, wn);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qsum += __shfl_xor_sync(FULL, qsum, o);
  if (lane == 0) s_red[warp] = qsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tsum = 0ull;
    for (int w = 0; w < NORM_BLOCK / 32; ++w) tsum += s_red[w];
    atomicAdd(B.cdf_tile + tile, tsum);  // the newborn part of a mixed tile comes from k_birth
  }
}
__global__ void __launch_bounds__(NORM_BLOCK, 8) k_normalise_lidar(KParams P, DevBufs B) {
  normalise_lidar_body(P, B, blockIdx.x);
}

// ====================================================================================
// k_resample (Alg. 7, systematic): with joint inclusive fixed-point CDF Q, total W and one
// uniform offset u in [0, W), output i takes the first source j with Q_j * nu > i W + u,
// that is the first j with Q_j > theta_i = floor((i W + u) / nu) (see theta_at).  A block
// takes a tile of 2048 sources: its inclusive CDF goes to shared memory, and its outputs
// [#{i : theta_i < E}, #{i : theta_i < E'}) for the CDF E before and E' after the tile
// (two counts at the start of the block) each find their source by binary
// search in it -- the same work for every output whatever the weights are.  Sources are
// written to Bsrc in output order (coalesced): posterior particle i is the record of source
// Bsrc[i] with the equal weight W 2^-40 / nu (Eq. resampledParticleWeights), which the next
// prediction reads through the index.
// ====================================================================================
constexpr int RES_BLOCK = 256, RES_ITEMS = NORM_TILE / RES_BLOCK;  // sources per thread
constexpr int RES_RUN = 3;  // consecutive outputs per thread

// count_theta_below by a warp: the 32 indices around the binary32 estimate are tested at
// once (theta is non-decreasing, so the lanes below the count form a prefix); outside that
// window, the serial count
__device__ __forceinline__ uint32_t count_theta_below_warp(const Theta &T, unsigned long long X, float inv_w,
                                                           uint32_t lane) {
  if (X <= T.c) return 0u;  // warp-uniform
  const uint32_t nu = T.nu;
  const float est = __fmul_rn(__fmul_rn(u64_to_f32_approx(X - T.c), (float)nu), inv_w);
  const uint32_t i0 = !(est > 0.0f) ? 0u : (est >= (float)nu ? nu : (uint32_t)est);
  const uint32_t base = i0 > 16u ? i0 - 16u : 0u;
  const uint32_t cand = base + lane;
  const bool below = cand < nu && theta_at(T, cand) < X;
  const uint32_t k = (uint32_t)__popc(__ballot_sync(FULL, below));
  if ((k > 0u || base == 0u) && (k < 32u || base + 32u >= nu)) return base + k;
  uint32_t r = 0u;
  if (lane == 0u) r = count_theta_below(T, X, inv_w);
  return __shfl_sync(FULL, r, 0);
}

// first y in [lo, hi] with Q[y] > th, hi if there is none (Q non-decreasing)
__device__ __forceinline__ uint32_t first_above(const unsigned long long *Q, uint32_t lo, uint32_t hi,
                                                unsigned long long th) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (Q[mid] > th) hi = mid; else lo = mid + 1u;
  }
  return lo;
}

// the same over a whole tile, Q[0 .. NORM_TILE) (entries past the tile's last source repeat
// its Q, and some Q of the tile exceeds th): the count of entries <= th, by halving steps
// of fixed number without a loop branch
__device__ __forceinline__ uint32_t first_above_tile(const unsigned long long *Q, unsigned long long th) {
  static_assert((NORM_TILE & (NORM_TILE - 1)) == 0, "power-of-two tile");
  uint32_t y = 0u;
#pragma unroll
  for (uint32_t half = NORM_TILE / 2; half >= 1u; half >>= 1)
    if (Q[y + half - 1u] <= th) y += half;
  return y;
}

__device__ __forceinline__ void resample_body(const KParams &P, const DevBufs &B, uint32_t blk) {
  __shared__ unsigned long long s_Q[NORM_TILE];  // inclusive CDF at each source of the tile
  __shared__ unsigned long long s_wsum[RES_BLOCK / 32];
  __shared__ uint32_t s_o[2];
  const uint32_t tile = blk;
  const uint32_t base = tile * NORM_TILE, ntot = P.nu + P.nu_b;
  const unsigned long long Wt = B.ctl->W_total;
  if ((P.flags & 0x2u) != 0u || Wt == 0ull) {
    // no resampling: the persistent particles carry over in sorted order (POST_DIRECT)
    for (uint32_t i = base + threadIdx.x; i < min(base + NORM_TILE, P.nu); i += RES_BLOCK) {
      B.Bw[i] = B.wn[i];
      B.Bsrc[i] = i;
    }
    return;
  }
  const unsigned long long E = tile > 0 ? B.cdf_incl[tile - 1] : 0ull;
  const Theta T = theta_of(B.ctl, P.nu);
  // the tile's outputs [o_lo, o_hi): counted by two warps while the others load weights
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < 2u) {
    const unsigned long long X = warp == 0u ? E : B.cdf_incl[tile];
    const uint32_t cnt = count_theta_below_warp(T, X, B.ctl->inv_w, lane);
    if (lane == 0u) s_o[warp] = cnt;
  }
  // the thread's quantised weights and the tile's CDF
  const uint32_t j0 = base + threadIdx.x * RES_ITEMS;
  float w[RES_ITEMS];
  if (j0 + RES_ITEMS <= P.nu) {
    load_runf<RES_ITEMS>(B.wn, j0, P.nu, w);
  } else {
#pragma unroll
    for (int it = 0; it < RES_ITEMS; ++it) {
      const uint32_t j = j0 + it;
      w[it] = j < P.nu ? __ldg(B.wn + j) : (j < ntot ? __ldg(B.bw + (j - P.nu)) : 0.0f);
    }
  }
  unsigned long long q[RES_ITEMS], loc = 0ull;
#pragma unroll
  for (int it = 0; it < RES_ITEMS; ++it) {  // neighbours mostly share a cell and so a weight
    q[it] = (it > 0 && w[it] == w[it - 1]) ? q[it - 1] : q40(w[it]);
    loc += q[it];
  }
  unsigned long long inc = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(FULL, inc, o);
    if (lane >= (uint32_t)o) inc += t;
  }
  if (lane == 31) s_wsum[warp] = inc;
  __syncthreads();
  unsigned long long Q = E + inc - loc;
  for (uint32_t k = 0; k < warp; ++k) Q += s_wsum[k];
#pragma unroll
  for (int it = 0; it < RES_ITEMS; ++it) {
    Q += q[it];
    s_Q[threadIdx.x * RES_ITEMS + it] = Q;
  }
  __syncthreads();
  // every output of the tile has E <= theta < the tile's last Q, so the search ends inside
  const uint32_t nS = min((uint32_t)NORM_TILE, ntot - base);
  const uint32_t o_lo = s_o[0], o_hi = s_o[1];
  // a thread takes RES_RUN consecutive outputs: the first by binary search over the tile,
  // the next ones from theta_{x+1} = theta_x + a + [rem_x + b >= nu] and a forward scan
  // (an output's source is never before the previous output's), bounded, then a search
  for (uint32_t x0 = o_lo + RES_RUN * threadIdx.x; x0 < o_hi; x0 += RES_RUN * RES_BLOCK) {
    uint32_t rem;
    unsigned long long th = theta_at(T, x0, &rem);
    uint32_t y = min(first_above_tile(s_Q, th), nS - 1u);
    B.Bsrc[x0] = base + y;
#pragma unroll
    for (int k = 1; k < RES_RUN; ++k) {
      const uint32_t x = x0 + k;
      if (x >= o_hi) break;
      rem += T.b;  // < 2 nu
      th += T.a;
      if (rem >= T.nu) {
        rem -= T.nu;
        ++th;
      }
      int steps = 0;
      while (y < nS - 1u && s_Q[y] <= th && steps < 4) {
        ++y;
        ++steps;
      }
      if (s_Q[y] <= th) y = first_above(s_Q, y, nS - 1u, th);
      B.Bsrc[x] = base + y;
    }
  }
}
__global__ void __launch_bounds__(RES_BLOCK, 6) k_resample(KParams P, DevBufs B) {
  resample_body(P, B, blockIdx.x);
}

}  // namespace dog
