// Work units of the symmetric pair sums (FP32 and double-FP32): target blocks
// of SYM_TB consecutive nodes times source bodies j >= the block's first body,
// dealt in equal contiguous ranges to one wave of CTAs.
#pragma once

constexpr int SYM_TB = 512;   // targets per block

struct SymUnits {
  int U, G, ntb, ns;
  const int* off;          // [ntb + 1]: first unit of each target block
  const long long* roff;   // [ntb]: first value of each target block's reverse rows
  __device__ __forceinline__ int start(int c) const { return (int)(((long long)c * U) / G); }
  __device__ __forceinline__ int cta_of(int u) const {
    int c = (int)(((long long)u * G) / U);
    while (c + 1 < G && start(c + 1) <= u) c++;
    while (c > 0 && start(c) > u) c--;
    return c;
  }
  __device__ __forceinline__ int first_body(int tb) const { return (int)(((long long)tb * SYM_TB) / ns); }
};

// Source template of the symmetric FP32 pair sum as a launch parameter block
// (it lands in the constant bank, which every lane of a warp reads at the same
// address): per node q, float2 entries 6q + d = (-xi_d, -xi_d) and 6q + 3 + d =
// (wn_d, wn_d); padding nodes sit far away with zero weight.
constexpr int SYM_TPARAM_NODES = 520;   // 512 nodes per sphere, padded to a multiple of 5 (or 8)
struct __align__(16) SymTmplParam {
  float4 v[SYM_TPARAM_NODES * 3];
};
