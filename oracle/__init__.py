"""CPU oracle (test infrastructure only): see cbp_oracle.cpp and oracle.py."""
