// Host-side functions shared between the translation units of the library.
#pragma once

#include "rmg_internal.cuh"

namespace rmg {

void build_tiles(Level& L);
void set_geometry(Level& L, int dim, int nreg, const int* dims);
void build_groups(Ctx& c, Level& L, const uint8_t* dir_comp, const uint8_t* rmask,
                  DBuf<int>& count);
void layout_create(Ctx& c, Level& L, int dim, int nreg, const int* dims, const int64_t* g64,
                   int64_t ncomp, const uint8_t* dir);
void split_from_csr(Ctx& c, Level& L, int kind, int B, const int64_t* rowptr, const int64_t* col,
                    const double* val);
void comp_to_reg(Ctx& c, const Level& L, const double* comp, double* reg, bool zero_masked);
void reg_to_comp(Ctx& c, const Level& L, const double* reg, double* comp, int average);
void regional_apply(Ctx& c, const Level& L, const double* u, double* y, double* ypart);

}  // namespace rmg
