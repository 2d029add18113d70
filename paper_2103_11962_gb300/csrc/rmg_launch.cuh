// Launch helper shared by the translation units: phase A (region stencils, scalar or B x B
// blocks) and phase B (interface groups) with one epilogue.
#pragma once

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <type_traits>
#include <unordered_map>
#include <utility>

#include "rmg_kernels.cuh"

namespace rmg {

// Blocks of kTile threads of `kernel` that one SM keeps resident (at most 8), queried once per
// kernel. The 27-point half-plane sweeps need 40 registers a thread, so an SM holds 6 of their
// blocks: a grid of 8 per SM left its last quarter of blocks to a second, sparse wave, and
// sizing the grid by residency took the C3 sweep from 0.33 to 0.23 ms.
inline int resident_per_sm(const void* kernel) {
  static std::mutex m;
  static std::unordered_map<const void*, int> cache;
  std::lock_guard<std::mutex> lock(m);
  auto it = cache.find(kernel);
  if (it != cache.end()) return it->second;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kTile, 0) != cudaSuccess) {
    cudaGetLastError();
    b = 8;
  }
  b = std::max(1, std::min(b, 8));
  cache.emplace(kernel, b);
  return b;
}

// The same for a kernel with `smem` bytes of dynamic shared memory; also raises the kernel's
// dynamic shared memory limit, once per device (the attribute belongs to the device's context).
inline int resident_per_sm_smem(const void* kernel, int smem) {
  static std::mutex m;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  RMG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(m);
  const auto key = std::make_pair(kernel, dev);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int b = 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kTile, smem) != cudaSuccess) {
    cudaGetLastError();
    b = 1;
  }
  b = std::max(1, std::min(b, 8));
  cache.emplace(key, b);
  return b;
}

// kernel<<<one resident wave of blocks over `work` tiles, kTile>>>(args...) on st.
template <typename... P, typename... A>
void launch_resident(const Ctx& c, void (*kernel)(P...), int work, cudaStream_t st,
                     A&&... args) {
  const int g = persistent_grid(c, work, resident_per_sm((const void*)kernel));
  kernel<<<g, kTile, 0, st>>>(std::forward<A>(args)...);
}

// Phase B alone (scalar levels): one thread per copy of every interface group.
template <typename AT, class Epi>
void launch_groups(Ctx& c, const Level& L, const AT* y, Epi epi, cudaStream_t st) {
  if (!L.ngroups) return;
  const int gs = persistent_grid(c, (L.nslots + 255) / 256);
  k_groups<AT><<<gs, 256, 0, st>>>(L.nslots, L.sgrp.get(), L.gptr.get(), L.gslot.get(), y, epi);
  RMG_LAUNCHED();
}

// Phase A over `sweep` (a tuned tile list of L; the level's run tiles when null), then phase B.
// An FP32 sweep given half planes (see k_level0_fp32) and their asymmetry flag reads the half
// form while the flag is 0.
template <class Epi, typename CT, typename VT, typename AT>
void launch_stencil(Ctx& c, const Level& L, const CT* coef, const VT* u, AT* y, Epi epi,
                    cudaStream_t st, int* launches, cudaEvent_t ev0 = nullptr,
                    cudaEvent_t ev1 = nullptr, const Grid* sweep = nullptr,
                    const float* half = nullptr, const int* asym = nullptr) {
  Grid G = sweep ? *sweep : L.grid();
  // staged tiles copy 16-byte chunks: with an unaligned u or half-plane array the level's run
  // tiles take over
  if (G.lx == -3 && ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(half)) & 15))
    G = L.grid();
  const int gb = persistent_grid(c, G.ntiles);
  // external record nodes when capturing, so the events can be timed after a graph replay
  if (ev0) RMG_CUDA(cudaEventRecordWithFlags(ev0, st, g_capturing ? cudaEventRecordExternal : 0));
  bool done = false;
  if constexpr (std::is_same<CT, float>::value && std::is_same<VT, float>::value &&
                std::is_same<AT, float>::value) {
    if (half && L.B == 1 && G.lx == -3) {
      RMG_REQUIRE(asym != nullptr && L.kind == 27, RMG_ERR_STATE,
                  "staged sweeps need the half planes of a 27-point stencil");
      const int smem = kStSmemFloats * (int)sizeof(float);
      const auto kern = k_stencil_half27_staged<Epi>;
      const int g = persistent_grid(c, G.ntiles, resident_per_sm_smem((const void*)kern, smem));
      kern<<<g, kStX * kStY, smem, st>>>(G, coef, half, asym, u, L.mult.get(), y, epi);
      done = true;
    } else if (half && L.B == 1) {
      RMG_REQUIRE(asym != nullptr, RMG_ERR_STATE, "half planes without their flag");
      const int nt = G.ntiles;
      const uint8_t* mu = L.mult.get();
      switch (L.kind) {
        case 5: launch_resident(c, k_stencil_half<5, Epi>, nt, st, G, coef, half, asym, u, mu, y, epi); break;
        case 7: launch_resident(c, k_stencil_half<7, Epi>, nt, st, G, coef, half, asym, u, mu, y, epi); break;
        case 9: launch_resident(c, k_stencil_half<9, Epi>, nt, st, G, coef, half, asym, u, mu, y, epi); break;
        default: launch_resident(c, k_stencil_half<27, Epi>, nt, st, G, coef, half, asym, u, mu, y, epi); break;
      }
      done = true;
    }
  }
  RMG_REQUIRE(done || G.lx != -3, RMG_ERR_STATE, "staged tiles outside a half-plane sweep");
  if (done) {
  } else if (L.B == 1) {
    switch (L.kind) {
      case 5: k_stencil<5, CT, VT, AT><<<gb, kTile, 0, st>>>(G, coef, u, L.mult.get(), y, epi); break;
      case 7: k_stencil<7, CT, VT, AT><<<gb, kTile, 0, st>>>(G, coef, u, L.mult.get(), y, epi); break;
      case 9: k_stencil<9, CT, VT, AT><<<gb, kTile, 0, st>>>(G, coef, u, L.mult.get(), y, epi); break;
      default: k_stencil<27, CT, VT, AT><<<gb, kTile, 0, st>>>(G, coef, u, L.mult.get(), y, epi); break;
    }
  } else {
    RMG_REQUIRE(L.B == 3 && (L.kind == 27 || L.kind == 9), RMG_ERR_ARG,
                "block operators need 3 dofs per node and a 27- or 9-point stencil");
    if (L.kind == 27)
      k_bstencil<27, 3, CT, VT, AT><<<gb, kTile, 0, st>>>(G, coef, u, L.mult.get(), y, epi);
    else
      k_bstencil<9, 3, CT, VT, AT><<<gb, kTile, 0, st>>>(G, coef, u, L.mult.get(), y, epi);
  }
  RMG_LAUNCHED();
  if (ev1) RMG_CUDA(cudaEventRecordWithFlags(ev1, st, g_capturing ? cudaEventRecordExternal : 0));
  if (launches) ++*launches;
  if (L.ngroups) {
    if (L.B == 1) {
      launch_groups(c, L, y, epi, st);
    } else {
      const int gg = persistent_grid(c, (L.ngroups + 255) / 256);
      k_groups_b<AT><<<gg, 256, 0, st>>>(L.ngroups, L.B, L.n_r, L.gptr.get(), L.gslot.get(), y, epi);
      RMG_LAUNCHED();
    }
    if (launches) ++*launches;
  }
}

}  // namespace rmg
