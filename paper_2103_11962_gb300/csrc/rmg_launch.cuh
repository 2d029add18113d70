// Launch helper shared by the translation units: phase A (region stencils, scalar or B x B
// blocks) and phase B (interface groups) with one epilogue.
#pragma once

#include <type_traits>

#include "rmg_kernels.cuh"

namespace rmg {

// Phase B alone (scalar levels): one thread per copy of every interface group.
template <typename AT, class Epi>
void launch_groups(Ctx& c, const Level& L, const AT* y, Epi epi, cudaStream_t st) {
  if (!L.ngroups) return;
  const int gs = persistent_grid(c, (L.nslots + 255) / 256);
  k_groups<AT><<<gs, 256, 0, st>>>(L.nslots, L.sgrp.get(), L.gptr.get(), L.gslot.get(), y, epi);
  RMG_LAUNCHED();
}

// Phase A over `sweep` (a tuned tile list of L; the level's run tiles when null), then phase B.
// An FP32 sweep given half planes (see k_half_pack) and their asymmetry flag reads the half
// form while the flag is 0.
template <class Epi, typename CT, typename VT, typename AT>
void launch_stencil(Ctx& c, const Level& L, const CT* coef, const VT* u, AT* y, Epi epi,
                    cudaStream_t st, int* launches, cudaEvent_t ev0 = nullptr,
                    cudaEvent_t ev1 = nullptr, const Grid* sweep = nullptr,
                    const float* half = nullptr, const int* asym = nullptr) {
  const Grid G = sweep ? *sweep : L.grid();
  const int gb = persistent_grid(c, G.ntiles);
  // external record nodes when capturing, so the events can be timed after a graph replay
  if (ev0) RMG_CUDA(cudaEventRecordWithFlags(ev0, st, g_capturing ? cudaEventRecordExternal : 0));
  bool done = false;
  if constexpr (std::is_same<CT, float>::value && std::is_same<VT, float>::value &&
                std::is_same<AT, float>::value) {
    if (half && L.B == 1) {
      RMG_REQUIRE(asym != nullptr, RMG_ERR_STATE, "half planes without their flag");
      switch (L.kind) {
        case 5: k_stencil_half<5><<<gb, kTile, 0, st>>>(G, coef, half, asym, u, L.mult.get(), y, epi); break;
        case 7: k_stencil_half<7><<<gb, kTile, 0, st>>>(G, coef, half, asym, u, L.mult.get(), y, epi); break;
        case 9: k_stencil_half<9><<<gb, kTile, 0, st>>>(G, coef, half, asym, u, L.mult.get(), y, epi); break;
        default: k_stencil_half<27><<<gb, kTile, 0, st>>>(G, coef, half, asym, u, L.mult.get(), y, epi); break;
      }
      done = true;
    }
  }
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
