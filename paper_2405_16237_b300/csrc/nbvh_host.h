// Host helpers shared by the host and CUDA translation units of the library.
#pragma once
#include <stdint.h>

#include "../../include/nbvh.h"

namespace nbvh_host {
bool desc_valid(const nbvh_model_desc* d);
bool layout(const nbvh_model_desc* d, int32_t* res, int32_t* dense, int64_t* size, int64_t* offset,
            int64_t* total);
int64_t mlp_params(const nbvh_model_desc* d);
}  // namespace nbvh_host
