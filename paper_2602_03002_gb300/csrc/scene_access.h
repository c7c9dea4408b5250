// scene_access.h -- read-only view of a frozen scene's device data for entry points that live in
// other translation units than rpl_api.cpp.
#pragma once
#include <cuda_runtime.h>

#include "../../include/rpl.h"

namespace rpl {

struct SceneInputs {
    int device;
    int wide;   // 1: the terrain BVH uses the eight-wide quantised layout
    const float4 *tnodes, *ttris, *lnodes, *ltris, *link_root;
    int32_t lroot[RPL_MAX_LINKS];
};

// Fills `out` from a scene whose link meshes have been uploaded (frozen by rpl_view_create).
// Returns false for a null or unfrozen scene.
bool scene_inputs(const rpl_scene *s, SceneInputs *out);

// Records the message returned by rpl_last_error() and returns `st`.
rpl_status set_error(rpl_status st, const char *msg);

}  // namespace rpl
