"""CPU oracle of the PIC-MCC diode -- test infrastructure only.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's cpu_baseline /
reference leg may import this package.
"""
