// tdct_classes.h -- the r-classes for which the fused codec is compiled.
//
// A launch for retention r runs the smallest class R >= r: work for scan
// positions >= R is removed at compile time and the exact r is applied with
// the per-launch multipliers.  The list holds every r that closes a
// zig-zag anti-diagonal (1, 3, 6, 10, 15, 21, 28, 36, 45, 55, 64) plus the
// retentions 4, 8, 16 and 32 used by the workloads of §6.1.
#pragma once

#define TDCT_FOR_EACH_CLASS_A(X) X(1) X(3) X(4) X(6) X(8)
#define TDCT_FOR_EACH_CLASS_B(X) X(10) X(15) X(16)
#define TDCT_FOR_EACH_CLASS_C(X) X(21) X(28) X(32)
#define TDCT_FOR_EACH_CLASS_D(X) X(36) X(45) X(55) X(64)
#define TDCT_FOR_EACH_CLASS(X) \
  TDCT_FOR_EACH_CLASS_A(X) TDCT_FOR_EACH_CLASS_B(X) TDCT_FOR_EACH_CLASS_C(X) TDCT_FOR_EACH_CLASS_D(X)

namespace tdct {
inline int r_class(int r) {
  static const int kClasses[] = {1, 3, 4, 6, 8, 10, 15, 16, 21, 28, 32, 36, 45, 55, 64};
  for (int c : kClasses)
    if (r <= c) return c;
  return 64;
}
}  // namespace tdct
