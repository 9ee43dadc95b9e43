"""Stage-II iteration on the device (Sec. 5.4): render, objective (Eqs. 21-24), adjoint, Adam.
Argument marshalling only; every step runs in libexmesh's kernels."""
from __future__ import annotations

import math

import torch

from . import native as N

# per-channel ranges of the 8-channel material map (A, R, M in [0, 1], the normal map free)
MAP_LO = [0.0, 0.0, 0.0, 0.0, 0.0, -math.inf, -math.inf, -math.inf]
MAP_HI = [1.0, 1.0, 1.0, 1.0, 1.0, math.inf, math.inf, math.inf]
ENV_LO = [0.0, 0.0, 0.0]
ENV_HI = [math.inf, math.inf, math.inf]


class Stage2Optimizer:
    """Optimises FP32 material maps [Hm, Wm, 8] and an environment map [He, We, 3] with a
    Renderer's fixed mesh and cameras.  Hyperparameters default to the paper's Stage-II table:
    material lr 2.5e-3, environment lr 1.5e-2, lambda_ssim 0.2, lambda_mat = lambda_env = 0.1,
    lambda_chroma0 = 0.1 decaying linearly to 0 over `total_steps`."""

    def __init__(self, renderer, maps, env, lr_maps=2.5e-3, lr_env=1.5e-2, lambda_ssim=0.2, lambda_mat=0.1,
                 lambda_env=0.1, lambda_chroma0=0.1, total_steps=10000, optimize_env=True):
        assert maps.dtype == torch.float32 and env.dtype == torch.float32
        self.r = renderer
        self.maps, self.env = maps, env
        self.lr_maps, self.lr_env = lr_maps, lr_env
        self.lambda_ssim, self.lambda_mat, self.lambda_env = lambda_ssim, lambda_mat, lambda_env
        self.lambda_chroma0, self.total_steps = lambda_chroma0, total_steps
        self.optimize_env = optimize_env
        dev = maps.device
        self.m_maps, self.v_maps = torch.zeros_like(maps), torch.zeros_like(maps)
        self.m_env, self.v_env = torch.zeros_like(env), torch.zeros_like(env)
        self.grad_maps, self.grad_env = torch.zeros_like(maps), torch.zeros_like(env)
        self.grad_rgb = torch.empty(renderer.image_shape(), dtype=torch.float32, device=dev)
        self.image = torch.empty(renderer.image_shape(), dtype=torch.float32, device=dev)
        # [0] total image term, [1] log-L1, [2] D-SSIM, [3] L_mat, [4] L_env, [5] L_chroma
        self.loss = torch.zeros(8, dtype=torch.float32, device=dev)
        self.t = 0
        self.last_lambda_chroma = lambda_chroma0

    def lambda_chroma(self):
        return self.lambda_chroma0 * max(0.0, 1.0 - self.t / self.total_steps)

    def gradients(self, target, stream=None):
        """Forward render, the objective and its full gradient into grad_maps / grad_env."""
        r = self.r
        r.forward(self.maps, self.env, out=self.image, stream=stream)
        N.exm_image_loss(r.ctx, self.image, target, self.lambda_ssim, self.loss[0:3], self.grad_rgb, stream)
        self.grad_maps.zero_()
        self.grad_env.zero_()
        r.backward(self.maps, self.grad_rgb, self.grad_maps, self.grad_env, None, stream=stream)
        N.exm_material_tv(r.ctx, self.maps, r.frame, r.params.flags, self.lambda_mat, self.loss[3:4],
                          self.grad_maps, stream)
        self.last_lambda_chroma = self.lambda_chroma()
        N.exm_env_regularizers(r.ctx, self.env, self.lambda_env, self.last_lambda_chroma, self.loss[4:6],
                               self.grad_env, stream)

    def step(self, target, stream=None):
        """One Stage-II iteration; returns the device loss vector (see `loss`)."""
        self.gradients(target, stream)
        self.t += 1
        N.exm_adam_step(self.r.ctx, self.maps, self.grad_maps, self.m_maps, self.v_maps, self.lr_maps, self.t,
                        MAP_LO, MAP_HI, stream=stream)
        if self.optimize_env:
            N.exm_adam_step(self.r.ctx, self.env, self.grad_env, self.m_env, self.v_env, self.lr_env, self.t,
                            ENV_LO, ENV_HI, stream=stream)
        return self.loss

    def total_loss(self):
        """Eq. 22 from the last call's terms (host read)."""
        l = self.loss.cpu().tolist()
        return l[0] + self.lambda_mat * l[3] + self.lambda_env * l[4] + self.last_lambda_chroma * l[5]
