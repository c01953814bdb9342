// Panel width per size class of ht_reduce_batched, written by
// paper_1710_08538_gb300/tune_batched.py (the timing of one ht_reduce call per
// candidate width on pencils of each class, FP64 with Q and Z, on the GPU the
// library is built for).  Regenerate with:
//   python -m paper_1710_08538_gb300.tune_batched --write
#pragma once

// classes: orders up to HT_TUNED_NMAX[i] take panel width HT_TUNED_NB[i]
constexpr int HT_TUNED_CLASSES = 4;
constexpr int HT_TUNED_NMAX[HT_TUNED_CLASSES] = {128, 256, 512, 1 << 30};
constexpr int HT_TUNED_NB[HT_TUNED_CLASSES] = {32, 32, 32, 32};

inline int ht_tuned_nb(int n) {
  for (int i = 0; i < HT_TUNED_CLASSES; ++i)
    if (n <= HT_TUNED_NMAX[i]) return HT_TUNED_NB[i];
  return 32;
}
