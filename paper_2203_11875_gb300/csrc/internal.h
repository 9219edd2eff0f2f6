// Internal (non-ABI) entry points shared by the library's translation units.
#pragma once
#include "opf_handle.h"

namespace condipm {

int eval_impl(opf_handle* h, const double* x, const double* u, const double* lam, const double* y, bool derivs);
int factor_async(opf_handle* h);
int condense_async(opf_handle* h, const double* sig_u, const double* sig_x, const double* sig_s);
int factor_kred_async(opf_handle* h, double delta_w);
int kkt_solve_impl(opf_handle* h, const double* rhs, double* step, int k);
int read_status(opf_handle* h, int* info = nullptr);
double* workspace(opf_handle* h, size_t n);
int lagrangian_gradient(opf_handle* h, const double* lam, const double* y, double* out);
int powerflow_impl(opf_handle* h, const double* u, double* x, double tol, int max_iter, int* iters);

}  // namespace condipm
