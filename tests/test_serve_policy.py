"""The server's choice of which resident jobs advance in a round (host
logic, no GPU): the fill policy takes jobs in admission order while their
nodes fit in max(fill_nodes, (1 + ride) x the oldest job's nodes)."""
from paper_1705_10045_gb300 import serve


def _server(policy, fill_nodes, ride, sides):
    s = object.__new__(serve.Server)
    s.policy, s.fill_nodes, s.ride = policy, fill_nodes, ride
    s.resident = {}
    for slot, n in enumerate(sides):
        job = serve.Job(name=f"j{slot}", params=dict(nx=n, ny=n, nz=n), fields=lambda: None, steps=1)
        s.resident[slot * 3 + 1] = (job, 0)   # slot ids need not be contiguous
    return s


def test_all_policy_advances_every_resident_job():
    s = _server("all", 0, 0.0, [100, 20, 150])
    assert s._choose() == [1, 4, 7]


def test_fill_policy_lets_small_jobs_ride_with_the_oldest():
    # oldest 100^3 = 1e6 nodes; target max(0, 1.25e6): 20^3 and 50^3 fit, 150^3 waits
    s = _server("fill", 0, 0.25, [100, 150, 20, 50])
    assert s._choose() == [1, 7, 10]


def test_fill_policy_fills_the_gpu_when_the_oldest_is_small():
    # oldest 32^3; fill_nodes 8e6 admits 150^3 (3.4e6) and 160^3 (4.1e6), not 192^3 then
    s = _server("fill", 8_000_000, 0.25, [32, 150, 192, 160])
    assert s._choose() == [1, 4, 10]


def test_oldest_job_always_advances():
    s = _server("fill", 0, 0.0, [300, 10])
    assert s._choose()[0] == 1
