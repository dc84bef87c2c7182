// scene_host.h -- host-side checking of a scene description and its parameter
// bindings, and the BaseScene the kernels read (the scene and the map theta -> scene,
// Eq. 1's f(x, theta)). One definition for prdpt_scene_upload and the allocation-free
// prdpt_smoothed_grad_static, so the two accept exactly the same scenes.
#pragma once

#include <cmath>
#include <cstring>

#include "../../include/prdpt.h"
#include "internal.h"

namespace prdpt {

// Checks the scene and the D bindings and fills B (primitives in natural order, record
// slots grouped by type, camera basis computed in double and rounded to float).
// allow_texture: a single binding row (4, material, T) may stand for the T x T x 3 texel
// albedos (D = 3 T^2). Returns null on success, else a message naming the first problem.
inline const char* build_base_scene(const prdpt_scene_desc* sd, const prdpt_param_binding* binds, int D,
                                    bool allow_texture, BaseScene* B) {
    if (sd->n_prims < 1 || sd->n_prims > kMaxPrims) return "n_prims must be in 1..32";
    if (sd->n_mats < 1 || sd->n_mats > kMaxMats) return "n_mats must be in 1..32";
    const bool texture = allow_texture && D >= 1 && binds[0].kind == kBindTexture;
    if (texture) {
        const int m = binds[0].index, T = binds[0].component;
        if (m < 0 || m >= sd->n_mats) return "texture binding: material index out of range";
        if (T < 1 || T > kMaxTexRes) return "texture binding: resolution must be in 1..1024";
        if (D != 3 * T * T) return "texture binding: D must be 3 * resolution^2";
    } else if (D < 1 || D > kMaxD) {
        return allow_texture ? "D must be in 1..64 (or 3 T^2 for one texture binding)" : "D must be in 1..64";
    }
    if (!sd->prim_type || !sd->prim_mat || !sd->prim_geom || !sd->mat_type || !sd->mat_param || !sd->camera ||
        !sd->background)
        return "scene array is NULL";
    std::memset(B, 0, sizeof(*B));
    B->n_prims = sd->n_prims;
    B->n_mats = sd->n_mats;
    B->D = D;
    B->tex_mat = texture ? binds[0].index : -1;
    B->tex_res = texture ? binds[0].component : 0;
    for (int i = 0; i < sd->n_mats; ++i) {
        if (sd->mat_type[i] < 0 || sd->mat_type[i] > 2) return "bad material type";
        B->mat_type[i] = sd->mat_type[i];
        for (int q = 0; q < 8; ++q) B->mat_param[i][q] = sd->mat_param[8 * i + q];
    }
    bool emission_bound[kMaxMats] = {};
    for (int d = 0; d < (texture ? 0 : D); ++d) {
        const int k = binds[d].kind, idx = binds[d].index, comp = binds[d].component;
        if (k == kBindPos || k == kBindRadius) {
            if (idx < 0 || idx >= sd->n_prims) return "binding: primitive index out of range";
            if (k == kBindRadius && sd->prim_type[idx] != kSphere) return "binding: radius of a non-sphere";
        } else if (k == kBindAlbedo || k == kBindEmission) {
            if (idx < 0 || idx >= sd->n_mats) return "binding: material index out of range";
            if (k == kBindEmission) emission_bound[idx] = true;
        } else {
            return "binding: unknown kind";
        }
        if (k != kBindRadius && (comp < 0 || comp > 2)) return "binding: component must be 0..2";
        B->bind_kind[d] = k;
        B->bind_index[d] = idx;
        B->bind_comp[d] = (k == kBindRadius) ? 0 : comp;
    }
    int lights = 0;
    for (int i = 0; i < sd->n_prims; ++i) {
        const int t = sd->prim_type[i], m = sd->prim_mat[i];
        if (t < 0 || t > 2) return "bad primitive type";
        if (m < 0 || m >= sd->n_mats) return "primitive material out of range";
        const float* mp = &sd->mat_param[8 * m];
        const bool can_emit = mp[3] > 0.f || mp[4] > 0.f || mp[5] > 0.f || emission_bound[m];
        if (t == kBox && can_emit) return "emissive boxes are not supported";
        lights += can_emit ? 1 : 0;
        B->prim_type[i] = t;
        B->prim_mat[i] = m;
        for (int q = 0; q < 9; ++q) B->prim_geom[i][q] = sd->prim_geom[9 * i + q];
        B->n_sph += (t == kSphere);
        B->n_quad += (t == kQuad);
        B->n_box += (t == kBox);
    }
    if (lights > kMaxLights) return "more than 8 emitters";
    int next[3] = {0, B->n_sph, B->n_sph + B->n_quad};  // record slots grouped by type, stable
    for (int i = 0; i < sd->n_prims; ++i) B->prim_slot[i] = next[B->prim_type[i]]++;
    double eye[3], look[3], up[3];
    for (int q = 0; q < 3; ++q) {
        eye[q] = sd->camera[q];
        look[q] = sd->camera[3 + q];
        up[q] = sd->camera[6 + q];
    }
    double f[3] = {look[0] - eye[0], look[1] - eye[1], look[2] - eye[2]};
    const double fn = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fn > 0)) return "camera eye equals look-at";
    for (double& x : f) x /= fn;
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    const double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rn > 0)) return "camera up is parallel to the view direction";
    for (double& x : r) x /= rn;
    const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    for (int q = 0; q < 3; ++q) {
        B->eye[q] = float(eye[q]);
        B->fwd[q] = float(f[q]);
        B->right[q] = float(r[q]);
        B->up[q] = float(u[q]);
        B->bg[q] = sd->background[q];
    }
    const double vfov = sd->camera[9];
    if (!(vfov > 0 && vfov < 180)) return "field of view must be in (0, 180) degrees";
    B->tan_half = float(std::tan(0.5 * vfov * M_PI / 180.0));
    return nullptr;
}

}  // namespace prdpt
