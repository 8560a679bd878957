// Layouts of the opaque handles of the C ABI (include/tk.h).  Private to libtk: every translation
// unit that reaches into a handle (abi.cpp, noalloc.cu) includes this one definition.
#pragma once

#include <memory>

#include "tk_internal.hpp"

struct tk_ctx {
  tk::Ctx c;
};
struct tk_space {
  tk::Space s;
};
struct tk_tmap {
  std::shared_ptr<tk::Structure> st;
};
struct tk_plan {
  int kind = 0;  // 0 permute, 1 contract, 2 block SVD
  std::shared_ptr<tk::PermutePlan> perm;
  std::shared_ptr<tk::ContractPlan> con;
  std::shared_ptr<tk::SvdPlan> svd;
};
