// Private definition of the library context (shared by the C-ABI sources).
#pragma once

#include <string>

struct pcl_ctx {
    int device = 0;
    int num_sms = 0;
    std::string err;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int *d_err = nullptr;  // device error word set by kernels whose bounded waits ran out
    unsigned long long wait_ns = 0;  // limit of each bounded device-side wait (0: one second)
    // device work counters: [0] window tasks the exact scan counted, [1] tasks in its windows,
    // [2], [3] the same for the re-extraction pair kernel
    unsigned long long *d_stats = nullptr;
};
