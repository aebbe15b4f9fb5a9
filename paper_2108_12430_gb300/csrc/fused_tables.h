// Generated by paper_2108_12430_gb300/gen_fused_tables.py -- do not edit.
// Compile-time tables of the fused DeepClean kernel (k_fused.cu): per layer the
// tensor-core lowering (input buffer geometry, K-steps, per-step A-operand
// start and LBO in 16-byte units relative to the input buffer) and the weight
// chunking.  Steps are ordered so that the first `split` read only the
// outputs of the previous layer's first 32 accumulator columns (the MMAs
// can start once half the previous epilogue is done); order(i) is the host
// lowering's index of step i.  The host plan checks them against its own lowering.
#pragma once
#include <stdint.h>

namespace gw {
namespace fz {

struct L0 {
  static constexpr int transposed = 0, cin = 21, cout = 8, K = 7, stride = 1, pad = 3;
  static constexpr int J = 8, Q = 8, lgQ = 3, coutp = 8, lgcoutp = 3, npad = 64;
  static constexpr int G = 3, P = 8, lgP = 3, rows = 130, dmin = -1;
  static constexpr int n_steps = 21, step_bytes = 2048, sps = 6, n_chunks = 4, chunk0 = 0, split = 0;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[21] = {68157441, 68157442, 68157571, 68157572, 68157701, 68157702, 68157831, 68157961, 68158090, 68158091, 68158220, 68158221, 68158350, 68158351, 67617, 67747, 67877, 8522151, 68266, 68396, 68526};
    return t[i];
  }
  // step i issues the host lowering's step order(i)
  __host__ __device__ static constexpr int order(int i) {
    constexpr int t[21] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20};
    return t[i];
  }
};

struct L1 {
  static constexpr int transposed = 0, cin = 8, cout = 16, K = 7, stride = 2, pad = 3;
  static constexpr int J = 4, Q = 4, lgQ = 2, coutp = 16, lgcoutp = 4, npad = 64;
  static constexpr int G = 1, P = 8, lgP = 3, rows = 130, dmin = -1;
  static constexpr int n_steps = 7, step_bytes = 2048, sps = 6, n_chunks = 2, chunk0 = 4, split = 3;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[7] = {65537, 65667, 8519941, 8454665, 8454795, 8454925, 911};
    return t[i];
  }
  // step i issues the host lowering's step order(i)
  __host__ __device__ static constexpr int order(int i) {
    constexpr int t[7] = {0, 1, 2, 3, 4, 5, 6};
    return t[i];
  }
};

struct L2 {
  static constexpr int transposed = 0, cin = 16, cout = 32, K = 7, stride = 2, pad = 3;
  static constexpr int J = 2, Q = 2, lgQ = 1, coutp = 32, lgcoutp = 5, npad = 64;
  static constexpr int G = 2, P = 4, lgP = 2, rows = 130, dmin = -1;
  static constexpr int n_steps = 9, step_bytes = 2048, sps = 6, n_chunks = 2, chunk0 = 6, split = 5;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[9] = {34078721, 34078722, 34078850, 34078851, 34078852, 34078980, 34078981, 34079110, 34079111};
    return t[i];
  }
  // step i issues the host lowering's step order(i)
  __host__ __device__ static constexpr int order(int i) {
    constexpr int t[9] = {0, 1, 2, 3, 4, 5, 6, 7, 8};
    return t[i];
  }
};

struct L3 {
  static constexpr int transposed = 0, cin = 32, cout = 64, K = 7, stride = 2, pad = 3;
  static constexpr int J = 1, Q = 1, lgQ = 0, coutp = 64, lgcoutp = 6, npad = 64;
  static constexpr int G = 4, P = 2, lgP = 1, rows = 131, dmin = -2;
  static constexpr int n_steps = 14, step_bytes = 2048, sps = 6, n_chunks = 3, chunk0 = 8, split = 6;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[14] = {17170433, 17170957, 17170434, 17170958, 17170435, 17170959, 17170563, 17171087, 17170564, 17171088, 17170565, 17171089, 17170566, 17171090};
    return t[i];
  }
  // step i issues the host lowering's step order(i)
  __host__ __device__ static constexpr int order(int i) {
    constexpr int t[14] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13};
    return t[i];
  }
};

struct L4 {
  static constexpr int transposed = 1, cin = 64, cout = 32, K = 7, stride = 2, pad = 3;
  static constexpr int J = 1, Q = 2, lgQ = 1, coutp = 32, lgcoutp = 5, npad = 64;
  static constexpr int G = 8, P = 1, lgP = 0, rows = 131, dmin = -1;
  static constexpr int n_steps = 16, step_bytes = 2048, sps = 6, n_chunks = 3, chunk0 = 11, split = 8;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[16] = {8585216, 8585478, 8585217, 8585479, 8585218, 8585480, 8585219, 8585481, 8585740, 8586002, 8585741, 8586003, 8585742, 8586004, 8585743, 8586005};
    return t[i];
  }
  // step i issues the host lowering's step order(i)
  __host__ __device__ static constexpr int order(int i) {
    constexpr int t[16] = {0, 1, 4, 5, 8, 9, 12, 13, 2, 3, 6, 7, 10, 11, 14, 15};
    return t[i];
  }
};

struct L5 {
  static constexpr int transposed = 1, cin = 32, cout = 16, K = 7, stride = 2, pad = 3;
  static constexpr int J = 2, Q = 4, lgQ = 2, coutp = 16, lgcoutp = 4, npad = 64;
  static constexpr int G = 4, P = 2, lgP = 1, rows = 130, dmin = -1;
  static constexpr int n_steps = 10, step_bytes = 2048, sps = 6, n_chunks = 2, chunk0 = 14, split = 4;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[10] = {17039361, 17039881, 17039362, 17039882, 17039490, 17040010, 17039491, 17040011, 17039492, 17040012};
    return t[i];
  }
  // step i issues the host lowering's step order(i)
  __host__ __device__ static constexpr int order(int i) {
    constexpr int t[10] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9};
    return t[i];
  }
};

struct L6 {
  static constexpr int transposed = 1, cin = 16, cout = 8, K = 7, stride = 2, pad = 3;
  static constexpr int J = 4, Q = 8, lgQ = 3, coutp = 8, lgcoutp = 3, npad = 64;
  static constexpr int G = 2, P = 4, lgP = 2, rows = 130, dmin = -1;
  static constexpr int n_steps = 7, step_bytes = 2048, sps = 6, n_chunks = 2, chunk0 = 16, split = 4;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[7] = {34078721, 34078722, 34078851, 34078852, 34078981, 34079110, 34079111};
    return t[i];
  }
  // step i issues the host lowering's step order(i)
  __host__ __device__ static constexpr int order(int i) {
    constexpr int t[7] = {0, 1, 2, 3, 4, 5, 6};
    return t[i];
  }
};

struct L7 {
  static constexpr int transposed = 0, cin = 8, cout = 1, K = 7, stride = 1, pad = 3;
  static constexpr int J = 8, Q = 8, lgQ = 3, coutp = 1, lgcoutp = 0, npad = 32;
  static constexpr int G = 1, P = 8, lgP = 3, rows = 130, dmin = -1;
  static constexpr int n_steps = 7, step_bytes = 1024, sps = 12, n_chunks = 1, chunk0 = 18, split = 3;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[7] = {65537, 65667, 65797, 8520071, 66186, 66316, 66446};
    return t[i];
  }
  // step i issues the host lowering's step order(i)
  __host__ __device__ static constexpr int order(int i) {
    constexpr int t[7] = {0, 1, 2, 3, 4, 5, 6};
    return t[i];
  }
};

constexpr int kChunks = 19;

}  // namespace fz
}  // namespace gw
