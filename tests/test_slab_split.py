"""The slab decomposition a multi-GPU run of one eye would use, checked on
CPU with the oracle: two gloo ranks each own half of the columns plus one
halo column, swap the pre-collision populations of their edge columns once
per step (the only exchange the stencil needs: every link reaches one cell),
and step their own sub-grid.  Gathered, the populations equal the undivided
run bit for bit, with the interpolated cornea rule on (whose q < 1/2 branch
reads the post-collision state of the upstream cell, possibly across the
cut).  No GPU code is involved: every run here has one GPU, so the library
runs independent replicas per GPU, and this pins the exchange plan itself."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

NX, NY, ANGLE, STEPS = 96, 48, 40.0, 120


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _global_state():
    import oracle as O
    from paper_2102_12663_gb300 import workloads as W
    pp = W.eye_params(NY, tau=0.8, Ra=1e4, K_tm=0.05)
    pp.update(bouzidi=1)
    m, g = O.eye_mask(NX, NY, ANGLE)
    return O, m, g, pp, O.State(g, O.make_params(**pp), m)


def _sub_geom(O, g, lo, hi):
    sg = O.Geom()
    for name, _ in O.Geom._fields_:
        setattr(sg, name, getattr(g, name))
    sg.nx = hi - lo
    sg.inlet_lo = g.inlet_lo - lo  # the inflow profile runs along x
    sg.arc_xc = g.arc_xc - lo
    return sg


def _rank(rank, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    O, m, g, pp, full = _global_state()
    xs = NX // 2
    lo, hi = (0, xs + 1) if rank == 0 else (xs - 1, NX)   # own columns plus one halo column
    own = slice(0, xs) if rank == 0 else slice(1, hi - lo)
    sub_m = np.ascontiguousarray(m[:, lo:hi])
    st = O.State(_sub_geom(O, g, lo, hi), O.make_params(**pp), sub_m)
    nl = hi - lo
    st.f[:] = full.f.reshape(9, NY, NX)[:, :, lo:hi].reshape(9, -1)
    st.T[:] = full.T.reshape(4, NY, NX)[:, :, lo:hi].reshape(4, -1)
    send_col = xs - 1 if rank == 0 else 1          # edge column the neighbour needs
    recv_col = xs if rank == 0 else 0              # this rank's halo column
    peer = 1 - rank
    for _ in range(STEPS):
        f3, t3 = st.f.reshape(9, NY, nl), st.T.reshape(4, NY, nl)
        out = torch.from_numpy(np.concatenate([f3[:, :, send_col], t3[:, :, send_col]]).copy())
        inc = torch.empty_like(out)
        if rank == 0:
            dist.send(out, peer)
            dist.recv(inc, peer)
        else:
            dist.recv(inc, peer)
            dist.send(out, peer)
        f3[:, :, recv_col] = inc[:9].numpy()
        t3[:, :, recv_col] = inc[9:].numpy()
        st.step()
    f3, t3 = st.f.reshape(9, NY, nl), st.T.reshape(4, NY, nl)
    q.put((rank, f3[:, :, own].copy(), t3[:, :, own].copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_slabs_with_halo_exchange_equal_the_whole_grid():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = dict((r, (f, t)) for r, f, t in (q.get(timeout=300) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    O, m, g, pp, full = _global_state()
    full.run(STEPS)
    f = np.concatenate([parts[0][0], parts[1][0]], axis=2).reshape(9, -1)
    t = np.concatenate([parts[0][1], parts[1][1]], axis=2).reshape(4, -1)
    assert np.array_equal(f, full.f) and np.array_equal(t, full.T)
