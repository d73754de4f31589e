"""Convenience layer over the C-ABI binding: holds a context and a plan, allocates the
output tensors with torch on the context's device, and calls the library.  Argument
marshalling only; every step runs in the library's kernels."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import links as L


@dataclass
class DeviceBatch:
    n_joints: "object"  # torch int32 [B]
    adj: "object"       # torch uint8 [B, n, n], or None with nbr
    jtype: "object"     # torch int8  [B, n]
    pos: "object"       # torch float32/float64 [B, n, 2]
    nbr: "object" = None  # torch int32 [B, n]: the adjacency as neighbour bit masks

    @property
    def B(self):
        return int(self.n_joints.shape[0])


def to_device(batch, device="cuda", non_blocking=False, masks=False) -> DeviceBatch:
    """Copy a MechBatch (numpy) to torch tensors on `device`; with masks=True the
    adjacency goes as neighbour bit masks (a fifth of the bytes at n_max 20)."""
    import torch

    def t(a):
        x = torch.from_numpy(np.ascontiguousarray(a))
        return x.to(device, non_blocking=non_blocking)

    if masks:
        return DeviceBatch(t(batch.n_joints), None, t(batch.jtype), t(batch.pos), t(batch.masks().view(np.int32)))
    return DeviceBatch(t(batch.n_joints), t(batch.adj), t(batch.jtype), t(batch.pos))


@dataclass
class SimOut:
    valid: "object"
    lock_step: "object"
    min_disc: "object"
    traj: "object" = None
    path: "object" = None
    out_index: "object" = None
    n_out: "object" = None
    status: "object" = None
    row_offset: "object" = None  # packed rows: joint offset of each row (int64 [rows + 1])


class Simulator:
    """One context + one plan of fixed capacity on a CUDA device."""

    def __init__(self, capacity: int, n_max: int, device: int = 0, stream=None):
        import torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = L.links_create(device, self.stream)
        self.plan = L.links_plan_create(self.ctx, capacity, n_max)
        self.capacity, self.n_max = capacity, n_max
        self.B = 0

    def close(self):
        if self.plan is not None:
            L.links_plan_free(self.plan)
            self.plan = None
        if self.ctx is not None:
            L.links_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def build(self, db: DeviceBatch, status=None):
        """Device plan build; returns the status tensor (int32 [B])."""
        import torch
        if status is None:
            status = torch.empty(db.B, dtype=torch.int32, device=self.device)
        if db.nbr is not None:
            L.links_plan_build_masks(self.ctx, self.plan, db.n_joints, db.nbr, db.jtype, db.pos, status)
        else:
            L.links_plan_build(self.ctx, self.plan, db.n_joints, db.adj, db.jtype, db.pos, status)
        self.B = db.B
        return status

    def build_host(self, batch):
        """Host plan build from a MechBatch (numpy); returns statuses (numpy)."""
        st = np.empty(batch.B, np.int32)
        L.links_plan_build_host(self.ctx, self.plan, np.ascontiguousarray(batch.n_joints, np.int32),
                                np.ascontiguousarray(batch.adj, np.uint8), np.ascontiguousarray(batch.jtype, np.int8),
                                np.ascontiguousarray(batch.pos), st)
        self.B = batch.B
        return st

    def alloc(self, T: int, precision: int, out_mode: int, traj=True, path=True, out_capacity=None) -> SimOut:
        import torch
        B, nm, dev = max(self.B, self.capacity), self.n_max, self.device  # valid for any later build
        fdt = torch.float64 if precision == L.PLAIN_F64 else torch.float32
        rows = B if out_mode == L.OUT_FULL else (B if out_capacity is None else out_capacity)
        o = SimOut(valid=torch.empty(B, dtype=torch.uint8, device=dev),
                   lock_step=torch.empty(B, dtype=torch.int16, device=dev),
                   min_disc=torch.empty(B, dtype=torch.float32, device=dev))
        if traj:
            o.traj = torch.empty((rows, nm, T, 2), dtype=fdt, device=dev)
        if path:
            o.path = torch.empty((rows, T, 2), dtype=fdt, device=dev)
        if out_mode == L.OUT_VALID_ONLY:
            o.out_index = torch.empty(max(rows, 1), dtype=torch.int32, device=dev)
            o.n_out = torch.zeros(1, dtype=torch.int32, device=dev)
        return o

    def simulate(self, T: int, precision: int = L.MIXED, out_mode: int = L.OUT_FULL, out: SimOut | None = None,
                 traj=True, path=True, out_capacity=None) -> SimOut:
        if out is None:
            out = self.alloc(T, precision, out_mode, traj, path, out_capacity)
        cap = 0 if out.out_index is None else (out.traj.shape[0] if out.traj is not None else
                                               (out.path.shape[0] if out.path is not None else out.out_index.shape[0]))
        L.links_simulate(self.ctx, self.plan, T, precision, out_mode, out.traj, out.path, out.valid, out.lock_step,
                         out.min_disc, out.out_index, cap, out.n_out)
        return out

    def alloc_packed(self, T: int, precision: int = L.MIXED, out_capacity=None, traj_capacity=None,
                     traj=True, path=True) -> SimOut:
        """Outputs of simulate_packed: traj [traj_capacity, T, 2] (joint rows; by default
        out_capacity * n_max, room for any rows), path [out_capacity, T, 2], out_index,
        row_offset [out_capacity + 1] int64, n_out."""
        import torch
        o = self.alloc(T, precision, L.OUT_VALID_ONLY, traj=False, path=path, out_capacity=out_capacity)
        rows = o.out_index.shape[0]
        fdt = torch.float64 if precision == L.PLAIN_F64 else torch.float32
        if traj:
            tc = rows * self.n_max if traj_capacity is None else traj_capacity
            o.traj = torch.empty((tc, T, 2), dtype=fdt, device=self.device)
        o.row_offset = torch.empty(rows + 1, dtype=torch.int64, device=self.device)
        return o

    def simulate_packed(self, T: int, precision: int = L.MIXED, out: SimOut | None = None, traj=True, path=True,
                        out_capacity=None, traj_capacity=None) -> SimOut:
        """Valid rows with the trajectories packed by joint count (links_simulate_packed):
        row r's joint j at out.traj[out.row_offset[r] + j]."""
        if out is None:
            out = self.alloc_packed(T, precision, out_capacity, traj_capacity, traj, path)
        cap = out.row_offset.shape[0] - 1
        tc = 0 if out.traj is None else out.traj.shape[0]
        L.links_simulate_packed(self.ctx, self.plan, T, precision, out.traj, tc, out.path, out.valid, out.lock_step,
                                out.min_disc, out.out_index, out.row_offset, cap, out.n_out)
        return out

    def simulate_topology(self, topo, T: int, out_mode: int = L.OUT_FULL, out: SimOut | None = None, traj=True,
                          path=True, out_capacity=None, n_escaped=None) -> SimOut:
        """Mixed simulation with the screen of a topology-specialised kernel first
        (links_simulate_topology; topo from links_topo_create)."""
        if out is None:
            out = self.alloc(T, L.MIXED, out_mode, traj, path, out_capacity)
        cap = 0 if out.out_index is None else (out.traj.shape[0] if out.traj is not None else
                                               (out.path.shape[0] if out.path is not None else out.out_index.shape[0]))
        L.links_simulate_topology(self.ctx, self.plan, topo, T, out_mode, out.traj, out.path, out.valid,
                                  out.lock_step, out.min_disc, out.out_index, cap, out.n_out, n_escaped)
        return out

    def simulate_two_stage(self, T: int, T_low: int, out: SimOut | None = None, traj=True, path=True,
                           out_capacity=None, n_low_valid=None) -> SimOut:
        """Low-fidelity screen on T_low positions, confirmation on T of the survivors,
        valid rows out (links_simulate_two_stage)."""
        if out is None:
            out = self.alloc(T, L.MIXED, L.OUT_VALID_ONLY, traj, path, out_capacity)
        cap = out.traj.shape[0] if out.traj is not None else (out.path.shape[0] if out.path is not None else
                                                              out.out_index.shape[0])
        L.links_simulate_two_stage(self.ctx, self.plan, T, T_low, out.traj, out.path, out.valid, out.lock_step,
                                   out.min_disc, out.out_index, cap, out.n_out, n_low_valid)
        return out

    def sync(self):
        L.links_sync(self.ctx)
