"""lb_links_noalloc: boundary links without any allocation by the library.

Some callers cannot allocate device memory: a plug-in running inside a host
program that owns the device's memory pool, or a real-time loop that cannot
take the implicit synchronisation of cudaMalloc.  lb_links_noalloc serves them
from a fixed scratch array inside the library, with outputs in buffers the
caller owns.  This test calls it through the C ABI twice in a row (the second
call finds the first call's bitmap in the shared scratch) and checks each
result against the FP64 CPU oracle's links for the same pose (bit-exact: both
sides evaluate the inside test in the same FP64 operation order) and against
lb_get_links of a context holding the same particle.
"""
import pytest

from lb_inputs import axis_angle_quaternion, box, particle, random_quaternion, rng
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def test_noalloc_links_match_oracle_and_context_links_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2403_05443_gb300 import lbsph as L

    g = rng(77)
    cases = [
        (box(32, 28, 36, 1.0), particle((5.5, 3.0, 2.5), (10.3, 20.7, 30.1), random_quaternion(g))),
        # a smaller particle in a channel, across the periodic x boundary: the
        # scratch still holds the larger bitmap of the first call
        (box(24, 40, 20, 1.0, walls=1),
         particle((4.0, 3.0, 2.0), (1.2, 19.6, 10.9), axis_angle_quaternion((0.2, 1.0, -0.4), 1.1))),
    ]
    cap = 20000
    pairs = torch.full((2 * cap,), -1, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    c, _ = L.lb_lattice()
    for b, p in cases:
        L.lb_links_noalloc(p["semi"], p["q"], p["x"], b["nx"], b["ny"], b["nz"], b["walls"],
                           pairs.data_ptr(), cap, count.data_ptr(), L.current_stream())
        torch.cuda.synchronize()
        n = int(count.item())
        pr = pairs[: 2 * n].cpu().numpy().reshape(n, 2)
        got = {(int(a), int(d)) for a, d in pr}
        sim = L.Simulation([b], [[p]], max_semi=8)
        node, d = sim.links()
        want = {(int(a), int(k)) for a, k in zip(node, d)}
        sim.close()
        assert n == len(want) > 0
        assert got == want
        # the oracle's links, as (node, velocity vector)
        onode, ocv = O.Sim(b, [p], nthreads=4).links()
        want_o = {(int(a), tuple(int(v) for v in cv)) for a, cv in zip(onode, ocv)}
        assert {(a, tuple(int(v) for v in c[d])) for a, d in got} == want_o


def test_noalloc_rejects_particles_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    from paper_2403_05443_gb300 import lbsph as L

    pairs = torch.zeros(2, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(L.LBError) as e:
        L.lb_links_noalloc((30.0, 4.0, 4.0), (1, 0, 0, 0), (64, 64, 64), 128, 128, 128, 0,
                           pairs.data_ptr(), 1, count.data_ptr(), L.current_stream())
    assert e.value.status == 7   # LB_ECAPACITY: cube of 66 nodes > 64
