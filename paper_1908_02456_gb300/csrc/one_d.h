// Internal declarations of the one-dimensional stepper (abc1d.h): the FP64 host
// blocks of one end (one_d_setup.cpp) and the device driver (one_d.cu).
#pragma once

#include <complex>
#include <string>

#include "abc1d.h"

namespace abc {
namespace oned {

struct Mat2 {
    std::complex<double> v[2][2];
};

// The left end's blocks (the right end's are these with rows and columns reversed).
struct Blocks1D {
    int order = 0;
    Mat2 K{}, M{}, A{}, B{}, B1{}, B0{}, A1{}, A0{};
};

bool green5(double h, double s, std::complex<double> u[2], std::complex<double> b[2]);
bool k_block(double h, double s, Mat2& K);
int build_blocks(const abc1d_params& p, Blocks1D& out, std::string& err);
int check_params(const abc1d_params* p, std::string& err);

}  // namespace oned
}  // namespace abc
