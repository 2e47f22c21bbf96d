// Autotuner shared by the launchers: picks one of a kernel's implementation variants (all
// bit-identical in result) per shape class, by timing them on the call's own inputs.
#pragma once

#include <cuda_runtime.h>

#include <functional>

namespace glu {

enum { kTuneSearch = 0, kTuneApply = 1, kTuneKernels = 2 };

// Chooses the variant for `key` (five ints naming the shape class): a forced variant, else a
// cached choice, else (tuning on and `st` not capturing a graph) the fastest of run(0..n-1)
// timed on `st` (synchronous), else variant 0. run(v) launches variant v on st and returns a
// GLU status. Returns a GLU status; *chosen receives the variant.
int tune_choose(int kernel, const int key[5], int nvariants, const std::function<int(int)>& run,
                cudaStream_t st, int* chosen);

// ceil(log2(n)) for n >= 1: the size part of a shape class.
int tune_size_class(long long n);

// While an object of this type lives, tune_choose on this host thread never times variants (it
// takes a forced or cached choice, else variant 0): no events are created, nothing synchronises.
struct TuneTimingOff {
    TuneTimingOff();
    ~TuneTimingOff();
    TuneTimingOff(const TuneTimingOff&) = delete;
    TuneTimingOff& operator=(const TuneTimingOff&) = delete;
    bool prev;
};

}  // namespace glu
