"""The FP64 viscous operator keeps the primitives of its state between the
stages of a time step: each LSERK4 stage update stores those of the updated
state for the next stage's lifting, face and volume kernels, and an input
whose stored primitives are stale has them formed afresh.  The values are the
same bitwise either way, so every sequence of calls that makes them stale (a
new state, an evaluation on another state, a captured step replayed after a
new state) must reproduce a plain run bitwise."""
import pytest

from paper_2606_18927_gb300 import dg, inputs as I
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

# small cases of the curvilinear Taylor-Green box (Roe) and of the
# wall-modelled channel (body force, Reichardt law)
CASES = [("tgv_sine_n3", "tgv_sine_n7_48", 3, (3, 3, 2)), ("channel_n4", "channel_n5", 4, (3, 2, 2))]


def _setup(name, N, elems):
    wl = I.workload(name, N=N, elems=elems)
    x, w = dg.lgl_nodes(N)
    X = I.node_coordinates(wl.spec, x)
    nbr = I.connectivity(wl.spec)
    U0 = I.initial_state(wl, X)
    U1 = I.perturb(U0, rel=2e-2, seed=7)
    return wl, X, nbr, U0, U1


@pytest.mark.parametrize("label,name,N,elems", CASES)
def test_stored_primitives_any_call_sequence_bitwise(label, name, N, elems):
    torch = torch_cuda()
    wl, X, nbr, U0, U1 = _setup(name, N, elems)
    phys, opts = wl.phys, dict(surf_flux=wl.surf_flux, law=wl.law)
    spec = wl.spec
    d0 = torch.from_numpy(U0).cuda()
    d1 = torch.from_numpy(U1).cuda()

    def state(op):
        out = torch.empty_like(d0)
        op.get_state(out)
        return out

    # plain run: three steps with the time derivative of the state after the first
    a = dg.Operator(spec.N, X, nbr, phys, **opts)
    dt = a.time_step(0.5, d0)
    a.set_state(d0)
    a.rk_steps(0.0, dt, 1)
    ut_a = torch.empty_like(d0)
    a.time_derivative(ut_a)
    a.rk_steps(dt, dt, 1)
    ref = state(a)
    a.rk_steps(2 * dt, dt, 1)
    ref3 = state(a)

    # an evaluation on another state inside a step, an evaluation on the
    # state, a captured step, a plain step
    b = dg.Operator(spec.N, X, nbr, phys, **opts)
    b.set_state(d0)
    b.rk_stage(0, 0.0, dt)
    tmp = torch.empty_like(d0)
    b.time_derivative(tmp, d1)
    for s in range(1, 5):
        b.rk_stage(s, 0.0, dt)
    ut_b = torch.empty_like(d0)
    b.time_derivative(ut_b)
    b.rk_steps_graph(dt, dt, 1)
    out_b = state(b)
    b.rk_steps(2 * dt, dt, 1)
    out_b3 = state(b)

    # a new state over primitives of another evolution; a graph captured on
    # one state and replayed after a new one
    c = dg.Operator(spec.N, X, nbr, phys, **opts)
    c.set_state(d1)
    c.rk_steps(0.0, dt, 1)
    c.set_state(d0)
    c.rk_steps(0.0, dt, 2)
    out_c = state(c)
    c.set_state(d1)
    c.rk_steps_graph(0.0, dt, 1)
    c.set_state(d0)
    c.rk_steps_graph(0.0, dt, 2)
    out_g = state(c)
    torch.cuda.synchronize()
    for op in (a, b, c):
        op.check_status()
        op.close()
    print(label, "max |U| change over two steps", float((ref - d0).abs().max()))
    assert float((ref - d0).abs().max()) > 0.0
    if name == "channel_n5":
        # the wall-law Newton solves start from the previous evaluation's
        # solution, which differs between these call sequences: the results
        # then agree to the solver's tolerance, not bitwise
        def close(x, y):
            return all(float((x[v] - y[v]).abs().max()) <= 1e-12 * float(y[v].abs().max()) for v in range(5))
    else:
        close = torch.equal
    assert close(ut_b, ut_a)
    assert close(out_b, ref)
    assert close(out_b3, ref3)
    assert close(out_c, ref)
    assert close(out_g, ref)
