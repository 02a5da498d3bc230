// dog_common.cuh -- parameter blocks, buffer table and the bounded decoupled look-back
// used by the single-pass scans of the filter kernels.
#pragma once
#include <cstddef>
#include <cstdint>

namespace dog {

constexpr uint32_t FULL = 0xffffffffu;

// error bits latched in DevCtl::err
enum : uint32_t {
  ERR_TIMEOUT_SORT = 1u, ERR_TIMEOUT_SEG = 2u, ERR_TIMEOUT_CELL = 4u, ERR_TIMEOUT_NORM = 8u,
  ERR_INPUT = 16u, ERR_INTERNAL = 32u
};

// dynamic tile counters (reset every frame by k_tick)
enum : int { CTR_SORT0 = 0, CTR_SORT1, CTR_SORT2, CTR_SEG, CTR_CELL, CTR_NORM, CTR_COUNT = 8 };

// look-back status: (epoch << 2) | state
enum : uint32_t { ST_NONE = 0, ST_AGG = 1, ST_INCL = 2 };

// spin bound of every device-wide wait: 2^20 polls with a short sleep (about a second),
// after which the waiter latches an error bit and proceeds; a waiter that sees an error
// already latched gives up at once, so a failed frame drains quickly.
constexpr int SPIN_LIMIT = 1 << 20;

struct DevCtl {
  uint32_t frame;          // incremented by k_tick at the start of every step
  float dt;
  uint32_t err;
  uint32_t n_birth_cells;  // written by the last k_cell tile
  unsigned long long R_total;
  unsigned long long W_total;
  unsigned long long u_offset;
  unsigned long long ctr[CTR_COUNT];
  uint32_t pad[8];
};

struct KParams {
  int W, H;
  uint32_t C;
  float s;
  uint32_t nu, nu_b;
  float p_S, p_B, alpha, sigma_pos, sigma_vel, sigma_B, sensor_x, sensor_y;
  uint32_t seed_lo, seed_hi, flags;
  int passes, dbits;
  uint32_t radix;
  uint32_t tiles_sort, tiles_seg, tiles_cell, tiles_norm;
};

struct DevBufs {
  DevCtl *ctl;
  // persistent posterior particles (B) and predicted particles (A)
  float *Bx, *By, *Bvx, *Bvy, *Bw;
  float *Ax, *Ay, *Avx, *Avy, *Aw;
  uint32_t *key_pred, *key_t0, *val_t0, *key_t1, *val_t1, *key_sorted, *perm;
  float *wn;
  uint32_t *rsrc;  // record only
  // newborn particles
  float *bx, *by, *bvx, *bvy, *bw;
  uint32_t *bcell, *bassoc;  // record only
  // cells
  float *mF;
  float *zO, *zF, *pA, *zv, *sgv;
  float *mO, *rho_p, *rho_b, *pO, *mean_x, *mean_y, *var_x, *var_y, *cov;
  float *mpred, *muA, *muU, *paeff;
  unsigned long long *S, *A;
  uint32_t *tag, *cstart, *cend;
  uint32_t *bl_cell;
  unsigned long long *bl_R;
  // scratch of the single-pass scans
  uint32_t *hist;                                // [passes][2048]
  uint32_t *lb_sort;                             // [passes][tiles_sort][radix]
  uint32_t *seg_st; unsigned long long *seg_v;   // [tiles_seg], [tiles_seg][2 agg + 2 incl]
  uint32_t *cell_st; unsigned long long *cell_v; // [tiles_cell], [tiles_cell][2 agg + 2 incl]
  uint32_t *cdf_st; unsigned long long *cdf_v;   // [tiles_norm], [tiles_norm][1 agg + 1 incl]
  uint32_t *mom_st; unsigned long long *mom_v;   // [tiles_norm], [tiles_norm][5 agg + 5 incl]
};

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {
  return *reinterpret_cast<const volatile uint32_t *>(p);
}
__device__ __forceinline__ void st_volatile(uint32_t *p, uint32_t v) {
  *reinterpret_cast<volatile uint32_t *>(p) = v;
}
__device__ __forceinline__ unsigned long long ld_cg64(const unsigned long long *p) { return __ldcg(p); }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Publish a tile's N values under state st (ST_AGG or ST_INCL).  Aggregate and inclusive
// values live in separate slots (an inclusive publish never overwrites an aggregate a
// reader may be loading).  Values first, a device fence, then the status word, so that a
// reader that sees the status sees the values.
template <int N>
__device__ __forceinline__ void lb_publish(uint32_t *status, unsigned long long *vals, uint32_t tile,
                                           uint32_t epoch, uint32_t st, const unsigned long long (&v)[N]) {
  unsigned long long *slot = vals + (size_t)tile * (2 * N) + (st == ST_INCL ? N : 0);
#pragma unroll
  for (int k = 0; k < N; ++k) __stcg(slot + k, v[k]);
  __threadfence();
  st_volatile(status + tile, (epoch << 2) | st);
}

// Warp-cooperative decoupled look-back (one full warp calls it; the result is valid in
// every lane).  Walks the predecessors of `tile` in windows of 32, summing aggregates
// until the nearest predecessor that published an inclusive value.  A window waits until
// all its tiles have published; tiles are taken in launch order from an atomic counter,
// so every predecessor is resident and publishes without waiting on anything.  Each wait
// is bounded: on timeout the error bit is latched and the walk stops.
template <int N>
__device__ void lb_lookback(const uint32_t *status, const unsigned long long *vals, uint32_t tile,
                            uint32_t epoch, unsigned long long (&acc)[N], uint32_t *err,
                            uint32_t errbit) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < N; ++k) acc[k] = 0ull;
  long long base = (long long)tile - 1;
  while (base >= 0) {
    const long long pt = base - lane;
    uint32_t st = ST_INCL;  // before tile 0: an inclusive zero
    if (pt >= 0) {
      int spins = 0;
      for (;;) {
        const uint32_t w = ld_volatile(status + pt);
        if ((w >> 2) == epoch && (w & 3u) != ST_NONE) {
          st = w & 3u;
          break;
        }
        if (++spins > SPIN_LIMIT) {
          atomicOr(err, errbit);
          st = ST_INCL;
          break;
        }
        if ((spins & 255) == 0 && ld_volatile(err) != 0u) {
          st = ST_INCL;
          break;
        }
        __nanosleep(32);
      }
    }
    const uint32_t incl = __ballot_sync(FULL, st == ST_INCL);
    const int stop = incl ? (__ffs(incl) - 1) : 31;
    __threadfence();
    unsigned long long v[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      v[k] = 0ull;
      if (pt >= 0 && lane <= stop)
        v[k] = ld_cg64(vals + (size_t)pt * (2 * N) + (st == ST_INCL ? N : 0) + k);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(FULL, v[k], o);
      acc[k] += v[k];
    }
    if (incl) break;
    base -= 32;
  }
}

}  // namespace dog
