// Host-side pieces of the engine shared with the server (csrc/server.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tc_stream.h"

namespace tc {

struct HostLayer {
    int cout, cin, stride, leaky;
    std::vector<float> w;  // OIHW
    std::vector<float> b;
};

// One depthwise-separable refinement layer: depthwise 3x3 with dilation (bias, no
// activation), then pointwise 1x1 (bias, LeakyReLU if leaky).
struct HostSep {
    int cin, cout, dil, leaky;
    std::vector<float> dw;  // [cin][3][3]
    std::vector<float> db;  // [cin]
    std::vector<float> pw;  // [cout][cin]
    std::vector<float> pb;  // [cout]
};

struct HostNet {
    int levels = 0, radius = 0;
    std::vector<int> chans;
    int dec[4] = {0, 0, 0, 0};
    std::vector<HostLayer> layers;
    std::vector<HostSep> ref;  // refinement network after the level-2 estimator (TCW2), or empty
};

// Parses and shape-checks a TCW1 weight blob (layout in include/tc_stream.h).
bool parse_weights(const uint8_t *p, size_t n, HostNet &net, std::string &err);

// Device memory a stream of width x height holds (feature pyramids, estimator buffers,
// flows, state, weights, host-entry staging), from the same sizes the stream allocates;
// lanes > 0: a batch of that many lanes (tc_create_batch; no host-entry staging).
size_t stream_device_bytes(const HostNet &net, int width, int height, tc_precision prec, int fs = 1, int lanes = 0);

}  // namespace tc

// Records the error of a stream-less call (read back with tc_last_error(NULL)).
tc_status tc_record_error(tc_status code, const std::string &msg);

// Sets what tc_op_last_used_tensor_cores() reports (1: the last stage op ran on the tensor
// cores, 0: on the CUDA cores).
void tc_set_last_op_tensor_cores(int used);
