"""One solve split across ranks by slabs (a grid larger than one GPU).

The 2D DFT of Sec. II.D is the x transforms of every row followed by the y
transforms of every column; the operators of Sec. III act on each spectral
element alone.  So the solve shards as a slab decomposition:

  1. rows      rank r owns rows y in [y0_r, y1_r): x transforms of its rows
               (fs_rows_forward) give the half spectrum of those rows,
               x-frequency-major [nx/2+1][rows_r];
  2. exchange  all-to-all: rank r sends the x frequencies owned by rank q
               (a in [a0_q, a1_q), a contiguous block of its spectrum) to q;
               each rank then holds whole columns [cols_q][ny];
  3. columns   forward y transform, operator, inverse y transform of its
               columns (fs_columns_apply);
  4. exchange  the transposed all-to-all back: rank q returns to each r the
               rows y in [y0_r, y1_r) of its columns;
  5. rows      inverse x transforms of its rows (fs_rows_inverse).

No TMA multicast or peer memory access is involved: every remote slab is
received into local memory before the local kernels run.  The exchange uses
torch.distributed: all_to_all where the backend has it (NCCL), paired
point-to-point sends and receives otherwise (gloo).  `emulate` runs all ranks
in one process with the exchange done by copies, for a single GPU.

The local steps come from a backend object with rows_forward(f_slab),
columns_apply(a0, cols, op, D, c, t) and rows_inverse(spec_slab); Library
below is the GPU backend (this library's kernels).
"""

import torch


def partition(n, world):
    """Near-even split of range(n) into `world` contiguous (start, count) parts."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(n, world)
    out, start = [], 0
    for r in range(world):
        cnt = base + (1 if r < extra else 0)
        out.append((start, cnt))
        start += cnt
    return out


def _exchange(send, recv, group=None):
    """recv[q] <- the tensor rank q sent to this rank (send[q] goes to rank q)."""
    import torch.distributed as dist

    rank = dist.get_rank(group)
    if dist.get_backend(group) == "nccl":
        dist.all_to_all(recv, send, group=group)
        return
    ops = []
    for q in range(len(send)):
        if q == rank:
            recv[q].copy_(send[q])
        else:
            ops.append(dist.P2POp(dist.isend, send[q], q, group))
            ops.append(dist.P2POp(dist.irecv, recv[q], q, group))
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()


def _as_real(x):
    return torch.view_as_real(x) if x.is_complex() else x


class Layout:
    """Row and x-frequency slabs of an nx x ny grid over `world` ranks."""

    def __init__(self, nx, ny, world):
        self.nx, self.ny, self.world = nx, ny, world
        self.rows = partition(ny, world)
        self.cols = partition(nx // 2 + 1, world)
        if any(c == 0 for _, c in self.rows) or any(c == 0 for _, c in self.cols):
            raise ValueError("more ranks than rows or x frequencies")


def _to_columns(spec_rows, lay, rank):
    """Blocks of this rank's row spectrum [nx/2+1][rows_r] for every rank's columns."""
    return [spec_rows[a0:a0 + na].contiguous() for a0, na in lay.cols]


def _from_rows(blocks, lay):
    """Whole columns [cols][ny] from the blocks [cols][rows_q] received from every rank."""
    return torch.cat(blocks, dim=1).contiguous()


def solve_rank(backend, lay, rank, f_slab, op, D=0.0, c=0.0, t=0.0, group=None):
    """This rank's part of one solve: f_slab [rows_r][nx] -> u_slab [rows_r][nx]."""
    y0, ny_r = lay.rows[rank]
    a0, na = lay.cols[rank]
    spec = backend.rows_forward(f_slab)                          # [nx/2+1][rows_r]
    send = _to_columns(spec, lay, rank)
    recv = [torch.empty((na, cnt), dtype=spec.dtype, device=spec.device) for _, cnt in lay.rows]
    _exchange([_as_real(x) for x in send], [_as_real(x) for x in recv], group)
    cols = _from_rows(recv, lay)                                 # [cols_r][ny]
    backend.columns_apply(a0, cols, op, D, c, t)
    send = [cols[:, y:y + cnt].contiguous() for y, cnt in lay.rows]
    recv = [torch.empty((cnt, ny_r), dtype=cols.dtype, device=cols.device) for _, cnt in lay.cols]
    _exchange([_as_real(x) for x in send], [_as_real(x) for x in recv], group)
    spec = torch.cat(recv, dim=0).contiguous()                  # [nx/2+1][rows_r]
    return backend.rows_inverse(spec)


def emulate(backend, f, world, op, D=0.0, c=0.0, t=0.0):
    """All ranks of a `world`-way sharded solve in one process (the exchanges
    become copies): f [ny][nx] -> u [ny][nx]."""
    ny, nx = f.shape
    lay = Layout(nx, ny, world)
    specs = [backend.rows_forward(f[y:y + cnt].contiguous()) for y, cnt in lay.rows]
    cols = []
    for q, (a0, na) in enumerate(lay.cols):
        c_q = torch.cat([s[a0:a0 + na] for s in specs], dim=1).contiguous()
        backend.columns_apply(a0, c_q, op, D, c, t)
        cols.append(c_q)
    out = []
    for r, (y, cnt) in enumerate(lay.rows):
        spec = torch.cat([c_q[:, y:y + cnt] for c_q in cols], dim=0).contiguous()
        out.append(backend.rows_inverse(spec))
    return torch.cat(out, dim=0)


class Library:
    """The local steps on this GPU through the library's slab entry points."""

    def __init__(self, plan, nx, ny, dtype, stream=None):
        from . import fsolve

        self.fs, self.plan, self.nx, self.ny, self.stream = fsolve, plan, nx, ny, stream
        self.real = torch.float32 if dtype == fsolve.FS_F32 else torch.float64
        self.cplx = torch.complex64 if dtype == fsolve.FS_F32 else torch.complex128

    def rows_forward(self, f_slab):
        nrows = f_slab.shape[0]
        spec = torch.empty((self.nx // 2 + 1, nrows), dtype=self.cplx, device=f_slab.device)
        self.fs.fs_rows_forward(self.plan, nrows, f_slab, spec, self.stream)
        return spec

    def columns_apply(self, a0, cols, op, D, c, t):
        ops = {"poisson": self.fs.FS_OP_POISSON, "diffusion": self.fs.FS_OP_DIFFUSION, "wave": self.fs.FS_OP_WAVE}
        self.fs.fs_columns_apply(self.plan, a0, cols.shape[0], ops[op], cols, D=D, c=c, t=t, stream=self.stream)

    def rows_inverse(self, spec):
        nrows = spec.shape[1]
        u = torch.empty((nrows, self.nx), dtype=self.real, device=spec.device)
        self.fs.fs_rows_inverse(self.plan, nrows, spec, u, self.stream)
        return u
