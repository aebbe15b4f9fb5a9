// Generated by paper_2108_12430_gb300/gen_fused_tables.py -- do not edit.
// Compile-time tables of the fused DeepClean kernel (k_fused.cu): per layer the
// tensor-core lowering (input buffer geometry, K-steps, per-step A-operand
// start and LBO in 16-byte units relative to the input buffer) and the weight
// chunking.  The host plan checks them against its own lowering.
#pragma once
#include <stdint.h>

namespace gw {
namespace fz {

struct L0 {
  static constexpr int transposed = 0, cin = 21, cout = 8, K = 7, stride = 1, pad = 3;
  static constexpr int J = 8, Q = 8, lgQ = 3, coutp = 8, lgcoutp = 3, npad = 64;
  static constexpr int G = 3, P = 8, lgP = 3, rows = 136, dmin = -1;
  static constexpr int n_steps = 21, step_bytes = 2048, sps = 6, n_chunks = 4, chunk0 = 0;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[21] = {71303169, 71303170, 71303305, 71303306, 71303441, 71303442, 71303577, 71303713, 71303848, 71303849, 71303984, 71303985, 71304120, 71304121, 67713, 67849, 67985, 8915481, 68392, 68528, 68664};
    return t[i];
  }
};

struct L1 {
  static constexpr int transposed = 0, cin = 8, cout = 16, K = 7, stride = 2, pad = 3;
  static constexpr int J = 4, Q = 4, lgQ = 2, coutp = 16, lgcoutp = 4, npad = 64;
  static constexpr int G = 1, P = 8, lgP = 3, rows = 136, dmin = -1;
  static constexpr int n_steps = 7, step_bytes = 2048, sps = 6, n_chunks = 2, chunk0 = 4;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[7] = {65537, 65673, 8913169, 8847905, 8848041, 8848177, 953};
    return t[i];
  }
};

struct L2 {
  static constexpr int transposed = 0, cin = 16, cout = 32, K = 7, stride = 2, pad = 3;
  static constexpr int J = 2, Q = 2, lgQ = 1, coutp = 32, lgcoutp = 5, npad = 64;
  static constexpr int G = 2, P = 4, lgP = 2, rows = 136, dmin = -1;
  static constexpr int n_steps = 9, step_bytes = 2048, sps = 6, n_chunks = 2, chunk0 = 6;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[9] = {35651585, 35651586, 35651720, 35651721, 35651722, 35651856, 35651857, 35651992, 35651993};
    return t[i];
  }
};

struct L3 {
  static constexpr int transposed = 0, cin = 32, cout = 64, K = 7, stride = 2, pad = 3;
  static constexpr int J = 1, Q = 1, lgQ = 0, coutp = 64, lgcoutp = 6, npad = 64;
  static constexpr int G = 4, P = 2, lgP = 1, rows = 136, dmin = -2;
  static constexpr int n_steps = 14, step_bytes = 2048, sps = 6, n_chunks = 3, chunk0 = 8;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[14] = {17825793, 17826337, 17825794, 17826338, 17825795, 17826339, 17825928, 17826472, 17825929, 17826473, 17825930, 17826474, 17825931, 17826475};
    return t[i];
  }
};

struct L4 {
  static constexpr int transposed = 1, cin = 64, cout = 32, K = 7, stride = 2, pad = 3;
  static constexpr int J = 1, Q = 2, lgQ = 1, coutp = 32, lgcoutp = 5, npad = 64;
  static constexpr int G = 8, P = 1, lgP = 0, rows = 136, dmin = -1;
  static constexpr int n_steps = 16, step_bytes = 2048, sps = 6, n_chunks = 3, chunk0 = 11;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[16] = {8912896, 8913168, 8913440, 8913712, 8912897, 8913169, 8913441, 8913713, 8912898, 8913170, 8913442, 8913714, 8912899, 8913171, 8913443, 8913715};
    return t[i];
  }
};

struct L5 {
  static constexpr int transposed = 1, cin = 32, cout = 16, K = 7, stride = 2, pad = 3;
  static constexpr int J = 2, Q = 4, lgQ = 2, coutp = 16, lgcoutp = 4, npad = 64;
  static constexpr int G = 4, P = 2, lgP = 1, rows = 136, dmin = -1;
  static constexpr int n_steps = 10, step_bytes = 2048, sps = 6, n_chunks = 2, chunk0 = 14;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[10] = {17825793, 17826337, 17825794, 17826338, 17825928, 17826472, 17825929, 17826473, 17825930, 17826474};
    return t[i];
  }
};

struct L6 {
  static constexpr int transposed = 1, cin = 16, cout = 8, K = 7, stride = 2, pad = 3;
  static constexpr int J = 4, Q = 8, lgQ = 3, coutp = 8, lgcoutp = 3, npad = 64;
  static constexpr int G = 2, P = 4, lgP = 2, rows = 136, dmin = -1;
  static constexpr int n_steps = 7, step_bytes = 2048, sps = 6, n_chunks = 2, chunk0 = 16;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[7] = {35651585, 35651586, 35651721, 35651722, 35651857, 35651992, 35651993};
    return t[i];
  }
};

struct L7 {
  static constexpr int transposed = 0, cin = 8, cout = 1, K = 7, stride = 1, pad = 3;
  static constexpr int J = 8, Q = 8, lgQ = 3, coutp = 1, lgcoutp = 0, npad = 32;
  static constexpr int G = 1, P = 8, lgP = 3, rows = 136, dmin = -1;
  static constexpr int n_steps = 7, step_bytes = 1024, sps = 12, n_chunks = 1, chunk0 = 18;
  __host__ __device__ static constexpr uint32_t apack(int i) {
    constexpr uint32_t t[7] = {65537, 65673, 65809, 8913305, 66216, 66352, 66488};
    return t[i];
  }
};

constexpr int kChunks = 19;

}  // namespace fz
}  // namespace gw
