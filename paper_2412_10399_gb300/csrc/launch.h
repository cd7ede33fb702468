// Host-side launchers of the CK-MPM kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace ck {

struct LaunchCfg {
  cudaStream_t stream;
  int persistent_ctas;  // CTAs of the persistent P2G / update / G2P launches
  int sm_count = 1;     // SMs of the device (grid of the float64 pass)
  int g2p_minb = 4;     // resident G2P warps per SM / 4 the register budget targets
  int transfer = 0;     // 0 APIC + MLS, 1 PIC, 2 APIC with the kernel gradient
  int p2g_rep = 1;      // copies of the P2G shared accumulators (1 or 2)
  int p2g_rot = 0;      // one copy: components in the lane-rotated order (1) or in order (0)
  int p2g_fma = 0;      // APIC + MLS: fused-multiply-add rounding in blocks of >= 256 particles (1)
};

enum { LK_P2G = 0, LK_UPDATE = 1, LK_G2P = 2, LK_CLEAR = 3, LK_G2P_FP64 = 4, LK_G2P2G = 5, LK_LEFTOVER = 6 };

// transfer.cu
void launch_transfer(int kind, const LaunchCfg& lc, const StepView& v, int which);
void launch_read_particles(int kind, bool pic, cudaStream_t st, Pool P, const SceneDev* scenes, const MatDev* mats,
                           int scene, uint32_t start, uint32_t n, int field, float* out);
void launch_write_particles(bool pic, cudaStream_t st, Pool P, const SceneDev* scenes, const MatDev* mats, int scene,
                            uint32_t start, uint32_t n, int field, const float* in);
void launch_read_grid(int kind, cudaStream_t st, const StepView& v, int scene, int which, float* out);
void launch_admit(int kind, cudaStream_t st, Pool P, uint32_t* key, uint32_t* cnt, uint32_t* bnd,
                  const SceneDev* scenes, const MatDev* mats, int scene, uint32_t mat_base, uint32_t nmat,
                  uint32_t start, uint32_t n, const float* x, const float* v, const uint8_t* mat, const float* E,
                  uint32_t* err);
void launch_rekey(int kind, cudaStream_t st, Pool P, uint32_t* key, uint32_t* cnt, uint32_t* bnd,
                  const SceneDev* scenes, const MatDev* mats, uint32_t n, uint32_t* err);

// bin.cu
constexpr int kScanTile = 4096;  // keys per scan tile
struct BinScratch {
  uint32_t* tile_cnt;   // per tile: sum of counts
  uint32_t* tile_ne;    // per tile: non-empty keys
  const uint32_t* scene_tab;  // sorted (key_base, slot) pairs of alive scenes
  int n_scene_tab;
};
void launch_bin(cudaStream_t st, const StepView& v, const BinScratch& bs, int which, uint32_t n_gblocks,
                int grid_ctas);
enum { LB_SCAN_TILES = 0, LB_SCAN_TOP = 1, LB_SCAN_FINAL = 2, LB_SCATTER = 3, LB_GLIST = 4 };
void launch_mark_dead(cudaStream_t st, uint32_t* key, uint32_t start, uint32_t n);
void launch_table_reset(cudaStream_t st, uint32_t* table, const uint32_t* g_list, const uint32_t* n_g,
                        uint32_t pool_cap, int grid_ctas);

}  // namespace ck
