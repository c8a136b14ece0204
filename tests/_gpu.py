"""Device helpers for the GPU tests: every compute step goes through the C ABI (libmf.so);
torch only allocates device memory and moves arrays."""
import numpy as np
import torch

import paper_2609_04534_gb300 as mf

GEOM = {
    "cart": (mf.MF_AFFINE, None),
    "stretch": (mf.MF_AFFINE, [2.0, 0, 0, 0, 0.5, 0, 0, 0, 1.5, 0, 0, 0]),
    "shear": (mf.MF_AFFINE, [1.0, 0.3, 0.0, 0.1, 1.2, -0.2, 0.0, 0.25, 0.9, 0.1, -0.2, 0.3]),
    "curved": (mf.MF_CURVED_SIN, None),
}
SHEAR_A = np.array([[1.0, 0.3, 0.0], [0.1, 1.2, -0.2], [0.0, 0.25, 0.9]])
SHEAR_B = [0.1, -0.2, 0.3]


def oracle_op(orc, nx, ny, nz, k, geom, cm, bc):
    if geom == "cart":
        return orc.Op(nx, ny, nz, k, orc.AFFINE, cm=cm, bc=bc)
    if geom == "stretch":
        return orc.Op(nx, ny, nz, k, orc.AFFINE, cm=cm, bc=bc, A=np.diag([2.0, 0.5, 1.5]))
    if geom == "shear":
        return orc.Op(nx, ny, nz, k, orc.AFFINE, cm=cm, bc=bc, A=SHEAR_A, b=SHEAR_B)
    return orc.Op(nx, ny, nz, k, orc.CURVED, cm=cm, bc=bc, amp=0.1)


class DevOp:
    """An mf operator with its device workspace (torch-owned)."""

    def __init__(self, nx, ny, nz, k, geom="cart", kind=mf.MF_LAPLACE, mass=1.0, precision=mf.MF_FP64,
                 bc=mf.MF_BC_NONE, stream=0):
        g, aff = GEOM[geom]
        self.mesh = mf.mf_mesh_create(nx, ny, nz, g, aff, 0.1)
        self.op = mf.mf_operator_create(self.mesh, k, kind, mass, precision, bc)
        self.info = mf.mf_operator_info(self.op)
        self.dtype = torch.float32 if precision == mf.MF_FP32 else torch.float64
        self.ws = torch.empty(max(self.info["workspace_bytes"], 256), dtype=torch.uint8, device="cuda")
        mf.mf_operator_setup(self.op, self.ws.data_ptr(), self.ws.numel(), stream)
        self.n_native = self.info["n_native"]
        self.n_unique = self.info["n_unique"]
        self.n_cw = self.info["n_cellwise"]

    def close(self):
        mf.mf_operator_destroy(self.op)
        mf.mf_mesh_destroy(self.mesh)

    def native_from_unique(self, xu: np.ndarray) -> torch.Tensor:
        u = torch.as_tensor(xu, dtype=self.dtype, device="cuda").contiguous()
        xn = torch.empty(self.n_native, dtype=self.dtype, device="cuda")
        mf.mf_scatter_unique(self.op, u.data_ptr(), xn.data_ptr())
        return xn

    def unique_from_native(self, xn: torch.Tensor) -> np.ndarray:
        u = torch.empty(self.n_unique, dtype=self.dtype, device="cuda")
        mf.mf_gather_unique(self.op, xn.data_ptr(), u.data_ptr())
        torch.cuda.synchronize()
        return u.double().cpu().numpy()

    def canonical_from_native(self, xn: torch.Tensor) -> np.ndarray:
        c = torch.empty(self.n_cw, dtype=self.dtype, device="cuda")
        mf.mf_from_native(self.op, xn.data_ptr(), c.data_ptr())
        torch.cuda.synchronize()
        return c.double().cpu().numpy()

    def apply(self, xn: torch.Tensor, split=False) -> torch.Tensor:
        y = torch.full((self.n_native,), float("nan"), dtype=self.dtype, device="cuda")
        (mf.mf_apply_split if split else mf.mf_apply)(self.op, xn.data_ptr(), y.data_ptr())
        return y

    def dot(self, a: torch.Tensor, b: torch.Tensor, split=0) -> float:
        sc = torch.empty(mf.mf_reduce_workspace_bytes(self.op), dtype=torch.uint8, device="cuda")
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        mf.mf_dot(self.op, a.data_ptr(), b.data_ptr(), out.data_ptr(), sc.data_ptr(), sc.numel(), split)
        torch.cuda.synchronize()
        return float(out.item())


def rel_max(a, ref):
    return float(np.abs(np.asarray(a) - np.asarray(ref)).max() / max(np.abs(ref).max(), 1e-300))
