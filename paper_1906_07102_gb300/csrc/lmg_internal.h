// Internal declarations shared by the translation units of liblmg.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "lmg.h"

namespace lmg {

// Thread-local error message; set_error returns the status for `return set_error(...)`.
int set_error(int status, const std::string& msg);
void clear_error();

// Table design parameters (Appendix A node counts).
constexpr int kNg = 32;
constexpr int kMg = 16;
constexpr int kMaxW = 16;

}  // namespace lmg

struct lmg_table {
  int W = 0;
  double x0 = 0.0;      // kept fraction (API convention)
  double x0p = 0.0;     // paper's x0 = x0 / 2
  int Ms = 0;           // oversample
  int interp = 1;
  int correction = 0;
  int iterations = 0;   // optimiser iterations for the final W
  double E = 0.0;       // integrated misfit at the optimum (NaN for caller tables)
  std::vector<double> h_nodes;  // Ng+1 values on [0, x0p]
  std::vector<double> C;        // (Ms+1) x W, row-major
};

namespace lmg {

// Table builder (host float64), table.cpp.
int build_least_misfit(int W, double x0p, int Ms, lmg_table* t);
// Correction factors h(x_p) at x_p = (p - n_image/2) / N from the (optionally
// float32-rounded) table function; table.cpp.
void correction_factors(const lmg_table* t, int64_t n_image, int64_t N, bool single_precision,
                        double* h_out);

}  // namespace lmg
