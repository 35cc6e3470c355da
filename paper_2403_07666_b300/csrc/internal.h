// Library-internal view of a coil handle for entry points that live outside
// coil_api.cu (they need the device descriptor, not the handle's layout).
#pragma once

#include "../../include/coil.h"
#include "common.cuh"

namespace cq {

struct CoilView {
    const CoilDev* host;     // host copy of the descriptor
    const CoilDev* dev;      // device copy of the descriptor
    int device;
    int n_sm;
};

// Fill *v for handle c; false for a null handle.
bool coil_view(const coil_t* c, CoilView* v);

// Set the text returned by coil_last_error and return st.
coil_status coil_set_error(coil_t* c, coil_status st, const char* msg);

}  // namespace cq
