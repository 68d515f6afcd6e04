// C ABI of the compression set-up (cells between two plates, no fluid) and
// of its adjoint: cf_plates_set, cf_relax, cf_plate_force, cf_tape_clear,
// cf_relax_adjoint, cf_adjoint_gradients, cf_force_jvp, cf_force_param_vjp.
//
// Relaxation steps (unit-mass vertices): v <- c v + dt (f_el + f_plate),
// y <- y + dt v. A recorded cf_relax call appends a tape entry and keeps
// device checkpoints of (y, v) every kTapeStride steps and at its end.
// cf_relax_adjoint reverses the last entry: it adds dL/dF * dF/dy to lambda_y
// (F = top-plate force at the end of that call), then, segment by segment from
// the last, restores the checkpoint, recomputes the segment's states, and
// walks it backwards with m = dt lambda_y + lambda_v:
//   lambda_y <- lambda_y + dt (J_el + J_plate) m, lambda_v <- c m,
// accumulating dt m . df/d(mu, kappa, w) per cell in double.
#include "ctx.h"

namespace {

constexpr int kTapeStride = 50;

void free_adjoint(cf_ctx *c) {
    for (auto *p : c->ckpt) cudaFree(p);
    c->ckpt.clear();
    c->ck_used = 0;
    c->tape.clear();
    ++c->tape_gen;
    dfree(c->vel_r);
    dfree(c->lam);
    dfree(c->lamv);
    dfree(c->mvec);
    dfree(c->jv);
    dfree(c->vtmp);
    dfree(c->seg);
    dfree(c->segv);
    dfree(c->grad);
    dfree(c->gtmp);
    dfree(c->pforce);
    dfree(c->dF);
    dfree(c->zlo);
    dfree(c->zhi);
    c->adj_V = c->adj_C = 0;
}

// Buffers sized for the current mesh (reallocated, and the tape dropped, when
// cells were added since).
cf_status ensure_adjoint(cf_ctx *c) {
    const int C = (int)c->cells.size();
    if (c->adj_V == c->V && c->adj_C == C) return CF_OK;
    std::vector<float> zlo = c->zlo_h, zhi = c->zhi_h;
    free_adjoint(c);
    CUDA_TRY(c, dalloc(&c->vel_r, c->V));
    CUDA_TRY(c, dalloc(&c->lam, c->V));
    CUDA_TRY(c, dalloc(&c->lamv, c->V));
    CUDA_TRY(c, dalloc(&c->mvec, c->V));
    CUDA_TRY(c, dalloc(&c->jv, c->V));
    CUDA_TRY(c, dalloc(&c->vtmp, c->V));
    CUDA_TRY(c, dalloc(&c->seg, (size_t)(kTapeStride + 1) * c->V));
    CUDA_TRY(c, dalloc(&c->segv, (size_t)(kTapeStride + 1) * c->V));
    CUDA_TRY(c, dalloc(&c->grad, 3 * (size_t)C));
    CUDA_TRY(c, dalloc(&c->gtmp, 3 * (size_t)C));
    CUDA_TRY(c, dalloc(&c->pforce, C));
    CUDA_TRY(c, dalloc(&c->dF, C));
    CUDA_TRY(c, dalloc(&c->zlo, C));
    CUDA_TRY(c, dalloc(&c->zhi, C));
    CUDA_TRY(c, cudaMemsetAsync(c->vel_r, 0, sizeof(float4) * c->V, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->lam, 0, sizeof(float4) * c->V, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->lamv, 0, sizeof(float4) * c->V, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->grad, 0, sizeof(double) * 3 * C, c->stream));
    c->adj_V = c->V;
    c->adj_C = C;
    if ((int)zlo.size() == C) {
        c->zlo_h = zlo;
        c->zhi_h = zhi;
        CUDA_TRY(c, cudaMemcpyAsync(c->zlo, zlo.data(), sizeof(float) * C, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(c->zhi, zhi.data(), sizeof(float) * C, cudaMemcpyHostToDevice, c->stream));
    } else {
        c->zlo_h.clear();
        c->zhi_h.clear();
    }
    return CF_OK;
}

cf_status upload_plates(cf_ctx *c, const std::vector<float> &zlo, const std::vector<float> &zhi) {
    CUDA_TRY(c, cudaMemcpyAsync(c->zlo, zlo.data(), sizeof(float) * zlo.size(), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->zhi, zhi.data(), sizeof(float) * zhi.size(), cudaMemcpyHostToDevice, c->stream));
    return CF_OK;
}

// forces at u into c->fv, then one damped step (u_in, v_in) -> (u_out, v_out)
cf_status relax_step(cf_ctx *c, const MeshView &m, const float4 *u_in, const float4 *v_in, float4 *u_out,
                     float4 *v_out, float dt, float cd, float kp) {
    CUDA_TRY(c, launch_tet_force(m, u_in, c->d_err, c->stream));
    CUDA_TRY(c, launch_gather_spread(m, u_in, nullptr, nullptr, c->d_err, c->stream));
    CUDA_TRY(c, launch_plate_step(m, u_in, v_in, c->fv, u_out, v_out, dt, cd, kp, c->zlo, c->zhi, c->d_err,
                                  c->stream));
    return CF_OK;
}

cf_status save_state(cf_ctx *c, float4 *dst, const float4 *u, const float4 *v) {
    CUDA_TRY(c, cudaMemcpyAsync(dst, u, sizeof(float4) * c->V, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(dst + c->V, v, sizeof(float4) * c->V, cudaMemcpyDeviceToDevice, c->stream));
    return CF_OK;
}

cf_status need_cells(cf_ctx *c) {
    if (!c) return CF_EINVAL;
    if (c->T == 0) return fail(c, CF_ESTATE, "no cells");
    return ensure_adjoint(c);
}

// The parameter gradients are per cell: a cell whose tets carry their own
// materials has no single (mu, kappa, w) to differentiate.
cf_status need_uniform_materials(cf_ctx *c) {
    for (size_t i = 0; i < c->cells.size(); ++i)
        if (c->cells[i].per_tet)
            return fail(c, CF_ESTATE, "cell %zu has per-tet materials: parameter gradients are per cell", i);
    return CF_OK;
}

}  // namespace

extern "C" {

cf_status cf_plates_set(cf_ctx *c, double k_plate, const double *z_lo, const double *z_hi) {
    cf_status st = need_cells(c);
    if (st != CF_OK) return st;
    DeviceGuard dg(c->device);
    const int C = (int)c->cells.size();
    if (!z_lo || !z_hi || !(k_plate >= 0.0) || !std::isfinite(k_plate)) return fail(c, CF_EINVAL, "bad plates");
    std::vector<float> lo(C), hi(C);
    for (int i = 0; i < C; ++i) {
        if (!(std::isfinite(z_lo[i]) && std::isfinite(z_hi[i]) && z_lo[i] < z_hi[i]))
            return fail(c, CF_EINVAL, "cell %d: need finite plates with z_lo < z_hi", i);
        lo[i] = (float)z_lo[i];
        hi[i] = (float)z_hi[i];
    }
    c->k_plate = (float)k_plate;
    c->zlo_h = lo;
    c->zhi_h = hi;
    st = upload_plates(c, lo, hi);
    return st != CF_OK ? st : wait_stream(c);
}

cf_status cf_relax(cf_ctx *c, int32_t n, double dt, double damping, int32_t record) {
    cf_status st = need_cells(c);
    if (st != CF_OK) return st;
    DeviceGuard dg(c->device);
    if ((int)c->zlo_h.size() != (int)c->cells.size()) return fail(c, CF_ESTATE, "call cf_plates_set first");
    if (n < 1 || !(dt > 0.0) || !std::isfinite(dt)) return fail(c, CF_EINVAL, "need n >= 1 and dt > 0");
    if (!(damping >= 0.0 && damping < 1.0)) return fail(c, CF_EINVAL, "need 0 <= damping < 1");
    const MeshView m = view(c);
    float4 *u = c->u[c->cur];
    const float cd = (float)damping;
    cf_ctx::TapeEntry e{};
    if (record) {
        e.n = n;
        e.dt = (float)dt;
        e.c = cd;
        e.kp = c->k_plate;
        e.zlo = c->zlo_h;
        e.zhi = c->zhi_h;
        e.ck0 = c->ck_used;
        e.nck = (n - 1) / kTapeStride + 2;
        for (const CellInfo &ci : c->cells) e.mats.push_back(ci.mat);
        while ((int)c->ckpt.size() < e.ck0 + e.nck) {
            float4 *p = nullptr;
            CUDA_TRY(c, dalloc(&p, 2 * (size_t)c->V));
            c->ckpt.push_back(p);
        }
    }
    for (int k = 0; k < n; ++k) {
        if (record && k % kTapeStride == 0) {
            st = save_state(c, c->ckpt[e.ck0 + k / kTapeStride], u, c->vel_r);
            if (st != CF_OK) return st;
        }
        st = relax_step(c, m, u, c->vel_r, u, c->vel_r, (float)dt, cd, c->k_plate);
        if (st != CF_OK) return st;
    }
    if (record) {
        st = save_state(c, c->ckpt[e.ck0 + e.nck - 1], u, c->vel_r);
        if (st != CF_OK) return st;
        c->ck_used = e.ck0 + e.nck;
        c->tape.push_back(e);
    }
    return consume_errors(c);
}

cf_status cf_plate_force(cf_ctx *c, double *out) {
    cf_status st = need_cells(c);
    if (st != CF_OK) return st;
    DeviceGuard dg(c->device);
    if (!out) return fail(c, CF_EINVAL, "null output");
    if ((int)c->zlo_h.size() != (int)c->cells.size()) return fail(c, CF_ESTATE, "call cf_plates_set first");
    const int C = (int)c->cells.size();
    CUDA_TRY(c, cudaMemsetAsync(c->pforce, 0, sizeof(double) * C, c->stream));
    CUDA_TRY(c, launch_plate_force(view(c), c->u[c->cur], c->k_plate, c->zlo, c->zhi, c->pforce, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(out, c->pforce, sizeof(double) * C, cudaMemcpyDeviceToHost, c->stream));
    return wait_stream(c);
}

cf_status cf_tape_clear(cf_ctx *c) {
    cf_status st = need_cells(c);
    if (st != CF_OK) return st;
    DeviceGuard dg(c->device);
    c->tape.clear();
    ++c->tape_gen;
    c->ck_used = 0;
    CUDA_TRY(c, cudaMemsetAsync(c->vel_r, 0, sizeof(float4) * c->V, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->lam, 0, sizeof(float4) * c->V, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->lamv, 0, sizeof(float4) * c->V, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->grad, 0, sizeof(double) * 3 * c->cells.size(), c->stream));
    return wait_stream(c);
}

cf_status cf_relax_adjoint(cf_ctx *c, const double *dF) {
    cf_status st = need_cells(c);
    if (st == CF_OK) st = need_uniform_materials(c);
    if (st != CF_OK) return st;
    DeviceGuard dg(c->device);
    if (c->tape.empty()) return fail(c, CF_ESTATE, "no recorded cf_relax call left to reverse");
    if (!dF) return fail(c, CF_EINVAL, "null dF");
    const cf_ctx::TapeEntry e = c->tape.back();
    const int C = (int)c->cells.size();
    for (int k = 0; k < C; ++k) {
        const float4 a = e.mats[k], b = c->cells[k].mat;
        if (a.x != b.x || a.y != b.y || a.z != b.z || a.w != b.w)
            return fail(c, CF_ESTATE, "cell %d: materials changed since the recorded cf_relax call", k);
    }
    const MeshView m = view(c);
    st = upload_plates(c, e.zlo, e.zhi);
    if (st != CF_OK) return st;
    CUDA_TRY(c, cudaMemcpyAsync(c->dF, dF, sizeof(double) * C, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, launch_adj_seed(m, c->ckpt[e.ck0 + e.nck - 1], e.kp, c->zlo, c->zhi, c->dF, c->lam, c->stream));
    for (int j = e.nck - 2; j >= 0; --j) {
        const int s0 = j * kTapeStride, len = std::min(kTapeStride, e.n - s0);
        const size_t V = (size_t)c->V;
        const float4 *ck = c->ckpt[e.ck0 + j];
        CUDA_TRY(c, cudaMemcpyAsync(c->seg, ck, sizeof(float4) * V, cudaMemcpyDeviceToDevice, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(c->segv, ck + V, sizeof(float4) * V, cudaMemcpyDeviceToDevice, c->stream));
        for (int i = 0; i + 1 < len; ++i) {  // states of the segment's steps
            st = relax_step(c, m, c->seg + i * V, c->segv + i * V, c->seg + (i + 1) * V, c->segv + (i + 1) * V, e.dt,
                            e.c, e.kp);
            if (st != CF_OK) return st;
        }
        for (int i = len - 1; i >= 0; --i) {
            const float4 *y = c->seg + i * V;
            CUDA_TRY(c, launch_adj_m(c->V, c->lam, c->lamv, e.dt, c->mvec, c->stream));
            CUDA_TRY(c, launch_force_jvp(m, y, c->mvec, c->jv, c->d_err, c->stream));
            CUDA_TRY(c, launch_param_vjp(m, y, c->mvec, (double)e.dt, c->grad, c->stream));
            CUDA_TRY(c, launch_adj_step(m, y, c->jv, c->mvec, c->lam, c->lamv, e.dt, e.c, e.kp, c->zlo, c->zhi,
                                        c->stream));
        }
    }
    c->tape.pop_back();
    c->ck_used = e.ck0;
    st = upload_plates(c, c->zlo_h, c->zhi_h);
    if (st != CF_OK) return st;
    return consume_errors(c);
}

cf_status cf_tape_generation(cf_ctx *c, int64_t *out) {
    if (!c || !out) return CF_EINVAL;
    *out = c->tape_gen;
    return CF_OK;
}

cf_status cf_adjoint_gradients(cf_ctx *c, double *out) {
    cf_status st = need_cells(c);
    if (st == CF_OK) st = need_uniform_materials(c);
    if (st != CF_OK) return st;
    DeviceGuard dg(c->device);
    if (!out) return fail(c, CF_EINVAL, "null output");
    CUDA_TRY(c, cudaMemcpyAsync(out, c->grad, sizeof(double) * 3 * c->cells.size(), cudaMemcpyDeviceToHost,
                                c->stream));
    return wait_stream(c);
}

cf_status cf_force_jvp(cf_ctx *c, const double *v, double *out) {
    cf_status st = need_cells(c);
    if (st != CF_OK) return st;
    DeviceGuard dg(c->device);
    if (!v || !out) return fail(c, CF_EINVAL, "null array");
    CUDA_TRY(c, cudaMemcpyAsync(c->stage, v, sizeof(double) * 3 * c->V, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, launch_pack3(c->stage, c->V, c->vtmp, c->stream));
    CUDA_TRY(c, launch_force_jvp(view(c), c->u[c->cur], c->vtmp, c->jv, c->d_err, c->stream));
    CUDA_TRY(c, launch_get_forces(c->jv, 0, c->V, c->stage, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(out, c->stage, sizeof(double) * 3 * c->V, cudaMemcpyDeviceToHost, c->stream));
    return consume_errors(c);
}

cf_status cf_force_param_vjp(cf_ctx *c, const double *lam, double *out) {
    cf_status st = need_cells(c);
    if (st == CF_OK) st = need_uniform_materials(c);
    if (st != CF_OK) return st;
    DeviceGuard dg(c->device);
    if (!lam || !out) return fail(c, CF_EINVAL, "null array");
    const int C = (int)c->cells.size();
    CUDA_TRY(c, cudaMemcpyAsync(c->stage, lam, sizeof(double) * 3 * c->V, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, launch_pack3(c->stage, c->V, c->vtmp, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->gtmp, 0, sizeof(double) * 3 * C, c->stream));
    CUDA_TRY(c, launch_param_vjp(view(c), c->u[c->cur], c->vtmp, 1.0, c->gtmp, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(out, c->gtmp, sizeof(double) * 3 * C, cudaMemcpyDeviceToHost, c->stream));
    return wait_stream(c);
}

}  // extern "C"

void cf_free_adjoint(cf_ctx *c) { free_adjoint(c); }
