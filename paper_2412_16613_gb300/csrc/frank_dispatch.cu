// frank_dispatch.cu -- tables of the per-K instantiations of the bit-sliced kernels
// (each built from frank_instance.cu, frank_trio_instance.cu or general_instance.cu with
// -DBITSSA_K=<K>).
#include "internal.h"

namespace bitssa {

#define BITSSA_FOR_EACH_K(X)                                                                     \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) \
  X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31)

#define BITSSA_DECLARE(k)                                                                      \
  int frank_launch_k##k(const FrankLaunch&, int, int, int, void*);                             \
  int frank_occupancy_k##k(int, int, int, int*);                                               \
  int frank_regs_k##k(int);                                                                    \
  int frank_trio_launch_k##k(const FrankLaunch&, int, int, void*);                             \
  int frank_trio_occupancy_k##k(int, int, int*);                                               \
  int frank_trio_regs_k##k(int);                                                               \
  int general_launch_k##k(const FrankLaunch&, int, int, int, void*);                           \
  int general_occupancy_k##k(int, int, int, int*);                                             \
  int general_regs_k##k(int);
BITSSA_FOR_EACH_K(BITSSA_DECLARE)

FrankLauncher frank_launcher(int K) {
  switch (K) {
#define BITSSA_CASE(k) \
  case k:              \
    return &frank_launch_k##k;
    BITSSA_FOR_EACH_K(BITSSA_CASE)
#undef BITSSA_CASE
    default:
      return nullptr;
  }
}

int frank_max_active_blocks(int K, int variant, int block, int smem, int* blocks) {
  switch (K) {
#define BITSSA_CASE(k) \
  case k:              \
    return frank_occupancy_k##k(variant, block, smem, blocks);
    BITSSA_FOR_EACH_K(BITSSA_CASE)
#undef BITSSA_CASE
    default:
      return -1;
  }
}

int frank_registers(int K, int variant) {
  switch (K) {
#define BITSSA_CASE(k) \
  case k:              \
    return frank_regs_k##k(variant);
    BITSSA_FOR_EACH_K(BITSSA_CASE)
#undef BITSSA_CASE
    default:
      return -1;
  }
}

FrankTrioLauncher frank_trio_launcher(int K) {
  switch (K) {
#define BITSSA_CASE(k) \
  case k:              \
    return &frank_trio_launch_k##k;
    BITSSA_FOR_EACH_K(BITSSA_CASE)
#undef BITSSA_CASE
    default:
      return nullptr;
  }
}

int frank_trio_max_active_blocks(int K, int variant, int smem, int* blocks) {
  switch (K) {
#define BITSSA_CASE(k) \
  case k:              \
    return frank_trio_occupancy_k##k(variant, smem, blocks);
    BITSSA_FOR_EACH_K(BITSSA_CASE)
#undef BITSSA_CASE
    default:
      return -1;
  }
}

int frank_trio_registers(int K, int variant) {
  switch (K) {
#define BITSSA_CASE(k) \
  case k:              \
    return frank_trio_regs_k##k(variant);
    BITSSA_FOR_EACH_K(BITSSA_CASE)
#undef BITSSA_CASE
    default:
      return -1;
  }
}

FrankLauncher general_launcher(int K) {
  switch (K) {
#define BITSSA_CASE(k) \
  case k:              \
    return &general_launch_k##k;
    BITSSA_FOR_EACH_K(BITSSA_CASE)
#undef BITSSA_CASE
    default:
      return nullptr;
  }
}

int general_max_active_blocks(int K, int variant, int block, int smem, int* blocks) {
  switch (K) {
#define BITSSA_CASE(k) \
  case k:              \
    return general_occupancy_k##k(variant, block, smem, blocks);
    BITSSA_FOR_EACH_K(BITSSA_CASE)
#undef BITSSA_CASE
    default:
      return -1;
  }
}

int general_registers(int K, int variant) {
  switch (K) {
#define BITSSA_CASE(k) \
  case k:              \
    return general_regs_k##k(variant);
    BITSSA_FOR_EACH_K(BITSSA_CASE)
#undef BITSSA_CASE
    default:
      return -1;
  }
}

}  // namespace bitssa
