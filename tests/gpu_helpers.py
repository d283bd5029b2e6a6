"""Helpers for the GPU tests: run the CUDA path through the C ABI and compare
with the oracle under the parity rule."""
import numpy as np

from paper_2507_09337_b300 import binding as B
from paper_2507_09337_b300 import workloads as wl


def rule12_error(G: np.ndarray, O: np.ndarray, nvar: int, extra_scale=None) -> float:
    """Largest |g - o| / max(|o|, s_v) over cells and variables, where s_v is the
    field's largest |momentum| for momentum components and |o| alone for rho
    and E (a plain relative error is meaningless where momentum is zero by
    symmetry). Arrays are block arrays [block, var, ...]. extra_scale (an
    array of the same shape) joins the per-cell maximum when given."""
    G = np.asarray(G)
    O = np.asarray(O)
    err = 0.0
    mom = np.abs(O[:, 1:nvar - 1]).max() if nvar > 2 else 0.0
    for v in range(nvar):
        o, g = O[:, v], G[:, v]
        scale = np.abs(o)
        if extra_scale is not None:
            scale = np.maximum(scale, np.abs(np.asarray(extra_scale)[:, v]))
        if 0 < v < nvar - 1:
            scale = np.maximum(scale, mom)
        d = np.abs(g - o)
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.where(d == 0, 0.0, d / scale)
        err = max(err, float(np.nanmax(r)) if r.size else 0.0)
        if not np.all(np.isfinite(g)):
            return float("inf")
    return err


def gpu_steps(spec, U0, nsteps, task=B.ORCHA_TASK_HYDRO_FP64, packets=None, tile=None, use_graph=False,
              record_dt=False):
    """Run nsteps on the GPU; returns (U, dts or None, device error word)."""
    import torch
    mesh = B.Mesh(spec, packets=packets)
    try:
        if tile is not None:
            mesh.set_tile(*tile)
        mesh.load(U0)
        dts = []
        stream = torch.cuda.current_stream()
        if record_dt:
            mesh.run(B.ORCHA_TASK_SIGNAL_SPEED)
            B.orcha_dt_reduce(mesh.handle)
            for _ in range(nsteps):
                dts.append(mesh.dt_value())
                mesh.run(B.ORCHA_TASK_GUARD_FILL)
                mesh.run(task)
                B.orcha_dt_reduce(mesh.handle)
                B.orcha_mesh_swap(mesh.handle)
        else:
            s = torch.cuda.Stream() if use_graph else stream
            s.wait_stream(stream)          # the load above was enqueued on the current stream
            with torch.cuda.stream(s):
                mesh.advance(nsteps, task, init_dt=True, use_graph=use_graph, stream=s)
            s.synchronize()
        err = mesh.poll()
        return mesh.store(), (np.array(dts) if record_dt else None), err
    finally:
        mesh.close()


def oracle_steps(oracle_mod, spec, U0, nsteps, rk2=False):
    m = oracle_mod.Mesh(**spec.oracle_kwargs())
    U, dts, _ = oracle_mod.run(m, U0, nsteps, rk2=rk2)
    return U, dts


def gpu_batch_steps(problems, nsteps, task=B.ORCHA_TASK_HYDRO_FP64, tile=(0, 0), use_graph=False, repeat=1):
    """Advance several meshes together through one batch (one persistent launch
    per step). problems: list of (spec, U0, packets or None). Returns the list
    of final states and the device error words."""
    import torch
    meshes = [B.Mesh(spec, packets=pk) for spec, _, pk in problems]
    batch = None
    try:
        for m, (_, U0, _) in zip(meshes, problems):
            m.load(U0)
        allp = [p for m in meshes for p in m.packets]
        batch = B.orcha_batch_create(allp, *tile)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        for r in range(repeat):
            B.orcha_batch_advance(batch, task, nsteps, r == 0, use_graph, s)
        s.synchronize()
        errs = [m.poll() for m in meshes]
        return [m.store() for m in meshes], errs
    finally:
        if batch:
            B.orcha_batch_destroy(batch)
        for m in meshes:
            m.close()


def _poll(mesh, stream=None):
    """Wait for the stream, then read and clear the mesh's device error word
    (returned, not raised)."""
    import ctypes
    word = ctypes.c_int32()
    B.lib().orcha_mesh_poll(mesh.handle, B._stream_ptr(stream), ctypes.byref(word))
    return word.value


def gpu_one_step(spec, U0, dt, task, tile, path):
    """One step (or stage) of `task` at a time step the caller gives (written
    into the mesh's dt_dev), through the packet path (guard fill + task, per
    stage for HYDRO_RK2) or one persistent batch launch with init_dt = 0.
    The device error word is read and cleared, not checked. Returns the new
    state."""
    import torch
    mesh = B.Mesh(spec)
    batch = None
    try:
        mesh.set_tile(*tile)
        mesh.load(U0)
        mesh.dt.fill_(dt)
        if path == "packet":
            if task == B.ORCHA_TASK_HYDRO_RK2:
                for st in (B.ORCHA_TASK_RK2_STAGE1, B.ORCHA_TASK_RK2_STAGE2):
                    mesh.run(B.ORCHA_TASK_GUARD_FILL)
                    mesh.run(st)
                    B.orcha_mesh_swap(mesh.handle)
            else:
                mesh.run(B.ORCHA_TASK_GUARD_FILL)
                mesh.run(task)
                B.orcha_mesh_swap(mesh.handle)
            _poll(mesh)
        else:
            batch = B.orcha_batch_create(mesh.packets, *tile)
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            B.orcha_batch_advance(batch, task, 1, False, False, s)
            _poll(mesh, s)
        return mesh.store()
    finally:
        if batch:
            B.orcha_batch_destroy(batch)
        mesh.close()


def gpu_batch_fixed_dt(spec, U0, dt, task, tile, nsteps):
    """nsteps steps of a batch task starting from the time step dt (written
    into dt_dev; init_dt = 0). Returns (state, device error word, dt_dev
    after the run)."""
    import torch
    mesh = B.Mesh(spec)
    batch = None
    try:
        mesh.load(U0)
        mesh.dt.fill_(dt)
        batch = B.orcha_batch_create(mesh.packets, *tile)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        B.orcha_batch_advance(batch, task, nsteps, False, False, s)
        err = _poll(mesh, s)
        return mesh.store(), err, mesh.dt_value()
    finally:
        if batch:
            B.orcha_batch_destroy(batch)
        mesh.close()
