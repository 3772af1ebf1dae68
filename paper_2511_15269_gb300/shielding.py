"""Active-shielding inverse design (Sec. III.B) on the GPU FMM.

Shield charges q_sh on a sphere are optimised so that the total potential of
external and shield charges is as uniform as possible on an inner sampling
sphere, while the shield's own potential on an outer sampling sphere stays
small (the loss of Sec. III.B):

    L_in  = sum_i (phi_i^(tot, in) - mean phi^(tot, in))^2
    L_out = sum_i (phi_i^(sh, out))^2
    L_reg = sum_i q_i^2
    L     = w_in L_in + w_out L_out + w_reg L_reg,  (w_in, w_out, w_reg) = (1, 0.2, 0.1)

Both potentials come from separate source/target trees (fmm_build_tree2);
gradients with respect to the shield charges flow through FMMPotential2,
whose backward pass evaluates the transposed problem on the reverse trees.
The optimiser is steepest descent with the exact step length of a quadratic
(the loss is quadratic in q_sh, Sec. III.B), the step taken from the change
of the gradient along the search direction.
"""
import torch

from . import fmm

WEIGHTS = (1.0, 0.2, 0.1)


class ShieldingProblem:
    """Trees and charges of one shielding geometry (see
    workloads.active_shielding for the layout of `geo`)."""

    def __init__(self, geo, p=8, leaf_size=16, theta=0.5, precision=fmm.FMM_FP32C, weights=WEIGHTS):
        dev = torch.device("cuda")
        as_dev = lambda a: torch.as_tensor(a, dtype=torch.float64).contiguous().to(dev)
        shield, ext = as_dev(geo["shield"]), as_dev(geo["ext"])
        inside, outside = as_dev(geo["inside"]), as_dev(geo["outside"])
        self.q_ext = as_dev(geo["q_ext"])
        self.n_sh = shield.shape[0]
        src_in = torch.cat([ext, shield]).contiguous()  # external charges first, then the shield
        args = (p, leaf_size, 2, theta, precision)
        self.t_in = fmm.fmm_build_tree2(src_in, inside, *args)
        self.r_in = fmm.fmm_build_tree2(inside, src_in, *args)
        self.t_out = fmm.fmm_build_tree2(shield, outside, *args)
        self.r_out = fmm.fmm_build_tree2(outside, shield, *args)
        self.weights = weights

    def potentials(self, q_sh):
        """(phi^(tot, in), phi^(sh, out)) for shield charges q_sh."""
        q_all = torch.cat([self.q_ext, q_sh])
        phi_in = fmm.FMMPotential2.apply(q_all, self.t_in, self.r_in)
        phi_out = fmm.FMMPotential2.apply(q_sh, self.t_out, self.r_out)
        return phi_in, phi_out

    def loss(self, q_sh):
        """Total loss and its three terms (L_in, L_out, L_reg)."""
        phi_in, phi_out = self.potentials(q_sh)
        l_in = ((phi_in - phi_in.mean()) ** 2).sum()
        l_out = (phi_out ** 2).sum()
        l_reg = (q_sh ** 2).sum()
        w_in, w_out, w_reg = self.weights
        return w_in * l_in + w_out * l_out + w_reg * l_reg, (l_in, l_out, l_reg)

    def grad(self, q_sh):
        q = q_sh.detach().clone().requires_grad_(True)
        total, _ = self.loss(q)
        (g,) = torch.autograd.grad(total, q)
        return g

    def optimise(self, steps, q0=None):
        """Steepest descent; returns the shield charges and the loss history."""
        q = torch.zeros(self.n_sh, dtype=torch.float64, device="cuda") if q0 is None else q0.clone()
        history = [float(self.loss(q)[0])]
        for _ in range(steps):
            g = self.grad(q)
            gg = float(torch.dot(g, g))
            if gg == 0.0:
                break
            hg = self.grad(q + g) - g  # Hessian times g: the gradient is affine in q
            ghg = float(torch.dot(g, hg))
            if ghg <= 0.0:
                break
            q = q - (gg / ghg) * g
            history.append(float(self.loss(q)[0]))
        return q, history

    def free(self):
        for t in (self.t_in, self.r_in, self.t_out, self.r_out):
            t.free()
