// dog_common.cuh -- parameter blocks, buffer table and small device helpers of the
// filter kernels.
#pragma once
#include <cstddef>
#include <cstdint>

namespace dog {

constexpr uint32_t FULL = 0xffffffffu;

// error bits latched in DevCtl::err
enum : uint32_t { ERR_INPUT = 16u, ERR_INTERNAL = 32u };

struct DevCtl {
  uint32_t frame;          // the last completed frame (advanced by the CDF scan, see this_frame)
  float dt;
  uint32_t err;
  uint32_t n_birth_cells;  // written by the newborn-mass tile scan
  unsigned long long R_total;
  unsigned long long W_total;
  unsigned long long u_offset;  // systematic resampling offset u in [0, W_total)
  float w_new;                   // resampled weight (W_total 2^-40) / nu
  float inv_w;                   // 1 / W_total (binary32 estimate for the output counts)
  uint32_t post_mode;            // posterior held as POST_RESAMPLED or POST_DIRECT
  // resampling thresholds theta_i = floor((i W + u) / nu) = i th_a + th_c +
  // floor((i th_b + th_e) / nu), from W = th_a nu + th_b and u = th_c nu + th_e
  unsigned long long th_a, th_c;
  uint32_t th_b, th_e;
  // ego motion applied at the start of this frame (filters created with the ego flag): the
  // vehicle moved by (ego_dx, ego_dy) m in the previous grid's axes and turned by the angle
  // whose cosine and sine are ego_c, ego_s, about the sensor position; ego_on = 0: none
  uint32_t ego_on;
  float ego_c, ego_s, ego_dx, ego_dy;
  // the frame whose radar velocity moments k_moments finishes: written by k_normalise,
  // which runs before the CDF scan advances the frame counter (k_moments runs beside it)
  uint32_t frame_mom;
};

// How the posterior particles are held between frames:
//   POST_RESAMPLED: particle i is the record of joint source Bsrc[i] (the sorted copy Os
//                   for a persistent source, the newborn records bs for a newborn one) and
//                   every weight is DevCtl::w_new;
//   POST_DIRECT:    particle i is Os[i] with weight Bw[i] (initial state, a restored
//                   checkpoint, or a frame without resampling).
enum : uint32_t { POST_RESAMPLED = 0, POST_DIRECT = 1 };

// Per-cell result of the segment pass, a 16-byte head read by the cell update for every
// cell: S = 2^-40 fixed-point sum of the predicted weights, tag = 2 frame (cell finished in
// one tile) or 2 frame + 1 (pieces in the accumulators).
struct __align__(16) CellSum {
  unsigned long long S;
  uint32_t tag;
  uint32_t pad;
};
static_assert(sizeof(CellSum) == 16, "cell head is 16 bytes");
// The lidar filter's compensated (double-float hi + lo) sums of w vx, w vy, w vx^2, w vy^2,
// w vx vy over a cell finished in one tile, 48 bytes (three 16-byte stores), read by the
// cell update only for such cells.
struct __align__(16) CellMom {
  float hi[5];
  float lo[5];
  uint32_t pad[2];
};
static_assert(sizeof(CellMom) == 48, "moment record is 48 bytes");

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
  // particle states are (x, y, vx, vy) records with the weight in a separate array:
  // predicted (A), predicted in sorted cell order (O), newborn (b); the posterior is
  // Bsrc / Bw over O and b (see post_mode)
  float4 *As, *Os, *bs;
  float *Bw, *Aw, *Ow, *bw;
  uint32_t *Bsrc;  // [nu] joint source of each posterior particle
  float4 *stage;   // [max(nu, nu_b)] staging for checkpoints and diagnostics
  uint32_t *key_pred, *key_t0, *val_t0, *key_t1, *val_t1, *key_sorted, *perm;
  float *wn;
  uint32_t *bcell, *bassoc;  // newborn cells and association flags (record only)
  // cells
  float *mF;
  const float *mF_in;  // [C] free mass the cell update starts from: mF, or for a filter with
                       // ego-motion compensation mF_warp (mF carried into the new grid)
  float *mF_warp;      // [C] (ego filters)
  float *rb_pred;      // [C] predicted newborn existence (the PHD/MIB filter, Sect. VI)
  // measurement grid.  DS filter: m_O, m_F (+ radar p_A, z_vr, sigma_vr).  PHD/MIB filter
  // (Bernoulli observation of Sect. VI): zO = z (1: a measurement occurred), zF = p_TP,
  // pA = p_A, zv = p_FP, sgv = p_c (clutter density; the single-object likelihood is 1)
  float *zO, *zF, *pA, *zv, *sgv;
  float *mO, *rho_p, *rho_b, *pO, *mean_x, *mean_y, *var_x, *var_y, *cov;
  float *mpred, *muA, *muU, *paeff;
  CellSum *csum;                   // [C] segment-pass result per cell
  CellMom *cmom;                   // [C] lidar moment sums of cells finished in one tile
  float *g_stage;                  // [5][C] measurement grid uploaded from the host
  float *c_stage;                  // [10][C] + error word: cells read back to the host
  unsigned long long *A;           // [C] fixed-point sum of g w (radar)
  uint32_t *cstart, *cend;         // [C] cell ranges (radar, or DOG_RECORD)
  uint32_t *bl_cell;               // [tiles_cell][1024] cells with newborn mass, per tile
  unsigned long long *bl_R;         // [tiles_cell][1024] tile-local inclusive newborn mass
  // all birth cells in cell order (entry G): first slot ([n + 1], last = nu_b), cell,
  // associated slots and the two newborn weights
  uint32_t *bl_first, *bl_gcell, *bl_nA;
  float *bl_wA, *bl_wUA;
  uint32_t *birth_block_entry;        // [ceil(nu_b / BIRTH_SLOTS) + 1] entry owning each slot block's first slot
  // scratch of the sort and the tile scans
  uint32_t *hist;                  // [passes][2048] digit histograms
  uint32_t *dcnt;                  // [passes][tiles_sort][radix] digit counts of each sort
                                   // tile, turned into global output offsets in place
  unsigned long long *S_piece, *A_piece;  // [C] pieces of cells spread over several tiles
  unsigned long long *Mx;          // [5][C] moment pieces of cells spread over several
                                   // normalisation tiles (radar filter)
  float *Pf;                       // [tiles_seg][2][10] lidar moment sums (hi[5], lo[5]) of
                                   // a segment tile's first segment begun earlier (or the
                                   // whole tile) and of its last segment continued later
  uint32_t *tile_whole;            // [tiles_seg] 1: the tile lies inside one cell
  uint32_t *cross_t1;              // [C] first segment tile of a cell spread over tiles
  unsigned long long *tile_q, *tile_qin;  // [tiles_cell] newborn mass per tile, inclusive
  uint32_t *tile_n, *tile_nin;             // [tiles_cell] birth cells per tile, inclusive
  unsigned long long *cdf_tile, *cdf_incl; // [tiles_norm] joint weight per tile, inclusive
  unsigned char *batch_slot;       // [1024] the filter's description for batched launches
};

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {
  return *reinterpret_cast<const volatile uint32_t *>(p);
}
__device__ __forceinline__ void st_volatile(uint32_t *p, uint32_t v) {
  *reinterpret_cast<volatile uint32_t *>(p) = v;
}

// The number of the frame being computed.  The control block holds the last completed
// frame: the joint-weight CDF scan advances it once it has drawn the frame's resampling
// offset.  Every other kernel that reads it runs before the scan (the newborn chain on the
// same stream, the normalisation joined in before it), except the radar filter's k_moments
// beside it, which reads the number that k_normalise kept (DevCtl::frame_mom).  Between
// frames it is the frame whose results the buffers hold.
__device__ __forceinline__ uint32_t this_frame(const DevCtl *ctl) { return ctl->frame + 1u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace dog
