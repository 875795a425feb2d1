"""torch.autograd wrapper of the spherical-cap sampler (reparameterised sampling).

``vndf_sample_autograd(wi_x, wi_y, wi_z, alpha_x, alpha_y, seed, counter_base,
stream_id, extended)`` returns (wm_x, wm_y, wm_z, pdf) from vndf_sample and, on
backward, calls vndf_sample_backward with the same Philox stream, so gradients
reach wi and alpha with the uniforms held fixed.  extended=True uses the cap
sampler's extended domain (incident directions below the horizon too).  Only the inputs and the three Philox
integers are saved; the backward kernel recomputes the forward in registers.
"""
import torch

from . import vndf_sample, vndf_sample_backward


class VndfSample(torch.autograd.Function):
    @staticmethod
    def forward(ctx, wi_x, wi_y, wi_z, alpha_x, alpha_y, seed, counter_base, stream_id, extended=False):
        wm_x, wm_y, wm_z, pdf = vndf_sample(wi_x, wi_y, wi_z, alpha_x, alpha_y, seed=seed,
                                            counter_base=counter_base, stream_id=stream_id,
                                            method="cap_extended" if extended else "cap")
        ctx.extended = extended
        ctx.isotropic = alpha_y is None
        ctx.save_for_backward(wi_x, wi_y, wi_z, alpha_x, *(() if alpha_y is None else (alpha_y,)))
        ctx.rng = (seed, counter_base, stream_id)
        return wm_x, wm_y, wm_z, pdf

    @staticmethod
    def backward(ctx, g_wm_x, g_wm_y, g_wm_z, g_pdf):
        saved = ctx.saved_tensors
        wi_x, wi_y, wi_z, alpha_x = saved[:4]
        alpha_y = None if ctx.isotropic else saved[4]
        seed, counter_base, stream_id = ctx.rng
        gw = [g_wm_x, g_wm_y, g_wm_z]
        if all(g is None for g in gw):
            gw = [None, None, None]
        else:
            gw = [torch.zeros_like(wi_x) if g is None else g.contiguous() for g in gw]
        need_wi = any(ctx.needs_input_grad[:3])
        need_alpha = ctx.needs_input_grad[3] or (not ctx.isotropic and ctx.needs_input_grad[4])
        gx, gy, gz, gax, gay = vndf_sample_backward(
            wi_x, wi_y, wi_z, alpha_x, alpha_y, seed=seed, counter_base=counter_base, stream_id=stream_id,
            g_wm_x=gw[0], g_wm_y=gw[1], g_wm_z=gw[2], g_pdf=None if g_pdf is None else g_pdf.contiguous(),
            want_wi=need_wi, want_alpha=need_alpha, extended=ctx.extended)
        return gx, gy, gz, gax, gay, None, None, None, None


def vndf_sample_autograd(wi_x, wi_y, wi_z, alpha_x, alpha_y=None, seed=0, counter_base=0, stream_id=0,
                         extended=False):
    return VndfSample.apply(wi_x, wi_y, wi_z, alpha_x, alpha_y, seed, counter_base, stream_id, extended)
